// Mesh-side kernels: charge assignment, diffusion smoothing, reductions, the
// Mass-Zero prediction / constraint residual / field update, the multigrid
// operators, and the force interpolation.  Mesh arrays are N^3, x fastest:
// index (iz*N + iy)*N + ix.  T is the bulk mesh type (double or float).
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace p3 {

// Sum of the six periodic neighbours of point (x, y, z).
template <typename T>
__device__ __forceinline__ T nb6(const T* __restrict__ f, int x, int y, int z, int n) {
    const int xm = x == 0 ? n - 1 : x - 1, xp = x == n - 1 ? 0 : x + 1;
    const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
    const int zm = z == 0 ? n - 1 : z - 1, zp = z == n - 1 ? 0 : z + 1;
    const int row = (z * n + y) * n;
    return f[row + xm] + f[row + xp] + f[(z * n + ym) * n + x] + f[(z * n + yp) * n + x] +
           f[(zm * n + y) * n + x] + f[(zp * n + y) * n + x];
}

// ---------------------------------------------------------------- assignment
// q_n = sum_a Q_a W(u_a - n): cubic B-spline charge assignment (Sec. 2,
// "charge assignment and smoothing"), deterministic and without atomics.
//
// A block owns a tile of kSpTX x kSpTY x kSpTZ mesh points and writes every
// point of it exactly once (no memset of q, no global atomics).  A particle
// at mesh coordinate u reaches the nodes floor(u)-1 .. floor(u)+2 per axis, so
// the tile [o, o+e) is reached only from u in [o-2, o+e+1): the block reads
// the cell-sorted particles of the cells covering that range (a superset:
// cell coordinate = u nc/n) in passes of kSpCap, keeps those with a node in
// the tile and sorts them stably by their first z node (a counting sort on
// 19 keys).  Warp w owns the tile planes 2w and 2w+1: it walks the particles
// whose z nodes reach those planes, in sorted order, one particle per warp
// instruction -- lane = (x node, y node, plane) -- and adds into its own
// planes of the shared-memory tile with plain loads and stores.  Every point
// is owned by one warp and receives its contributions in a fixed order, so
// the result is the same on every run, alone or in a batch.  The particles'
// tile-local nodes are precomputed per axis (-1 outside the tile), so
// periodic wrap needs no arithmetic in the accumulation; tiles of small
// meshes whose z nodes can alias (e + 3 > n) are walked in full by every warp.
constexpr int kSpTX = 32, kSpTY = 16, kSpTZ = 16;   // tile (8192 points)
constexpr int kSpRowP = kSpTX + 4;                  // padded row: the 4 y rows of a particle in distinct banks
constexpr int kSpPlaneP = kSpRowP * kSpTY + 16;     // padded plane: a warp's two planes in distinct banks
constexpr int kSpThreads = 256;                     // 8 warps x 2 planes
constexpr int kSpCap = 256;                         // candidate particles per pass (one per thread)
constexpr int kSpRows = 128;                        // cell rows per pass (2 segments each)
constexpr int kSpKeys = kSpTZ + 3;                  // first z node in [-3, kSpTZ - 1]

template <typename T>
struct SpEntry {
    int loc[3];   // per axis, byte k: tile-local node of weight k (signed), -1 outside the tile
    T w[3][4];    // weights; Q folded into the z weights
};

template <typename T>
inline size_t spread_smem_bytes() {
    return sizeof(T) * kSpPlaneP * kSpTZ + sizeof(SpEntry<T>) * kSpCap + sizeof(int) * 4 * kSpRows;
}

__device__ __forceinline__ int sp_loc(int packed, int k) { return (int)(signed char)(packed >> (8 * k)); }

__device__ __forceinline__ int imod(int v, int m) {
    const int r = v % m;
    return r < 0 ? r + m : r;
}

// Exclusive scan of one int per thread over a 1-D block of kSpThreads; the
// total is returned in *total (all threads).
__device__ __forceinline__ int sp_block_excl_scan(int v, int* total) {
    __shared__ int wtot[kSpThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wtot[wid] = incl;
    __syncthreads();
    int before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kSpThreads / 32; ++w) {
        const int t = wtot[w];
        before += w < wid ? t : 0;
        all += t;
    }
    __syncthreads();
    *total = all;
    return before + incl - v;
}

// Base node (wrapped) and weights of one particle: FP32 from the mesh
// coordinates of the mixed path, FP64 from the cell-ordered positions.
__device__ __forceinline__ void sp_particle(const MeshPt* __restrict__ src, int s, double, int, int b[3],
                                           float w[3][4]) {
    const MeshPt p = src[s];
    b[0] = p.bx;
    b[1] = p.by;
    b[2] = p.bz;
    bspline4f(p.tx, w[0]);
    bspline4f(p.ty, w[1]);
    bspline4f(p.tz, w[2]);
#pragma unroll
    for (int k = 0; k < 4; ++k) w[2][k] *= p.q;
}
__device__ __forceinline__ void sp_particle(const PQ* __restrict__ src, int s, double inv_h, int n, int b[3],
                                           double w[3][4]) {
    const PQ p = src[s];
    b[0] = bspline_axis(p.x, inv_h, n, w[0]);
    b[1] = bspline_axis(p.y, inv_h, n, w[1]);
    b[2] = bspline_axis(p.z, inv_h, n, w[2]);
#pragma unroll
    for (int k = 0; k < 4; ++k) w[2][k] *= p.w;
}

// The x segments (one, or two when the cell range wraps) of candidate cell
// row r (y, z cells) in cell order.
__device__ __forceinline__ void sp_row(const int* __restrict__ start, int nc, const int* cl, const int* nn, int r,
                                       int& b0, int& l0, int& b1, int& l1) {
    const int cy = imod(cl[1] + r % nn[1], nc), cz = imod(cl[2] + r / nn[1], nc);
    const int rb = (cz * nc + cy) * nc;
    const int x0 = imod(cl[0], nc);
    const int n0 = min(nn[0], nc - x0);
    b0 = start[rb + x0];
    l0 = start[rb + x0 + n0] - b0;
    b1 = start[rb];
    l1 = nn[0] > n0 ? start[rb + nn[0] - n0] - b1 : 0;
}

template <typename T, typename Src, bool VEC>
__global__ void __launch_bounds__(kSpThreads)
k_spread_tile(int n, int nc, const int* __restrict__ start, const Src* __restrict__ src, double inv_h,
              T* __restrict__ q) {
    extern __shared__ __align__(16) unsigned char sp_raw[];
    T* acc = reinterpret_cast<T*>(sp_raw);
    SpEntry<T>* ent = reinterpret_cast<SpEntry<T>*>(acc + kSpPlaneP * kSpTZ);
    int* seg_beg = reinterpret_cast<int*>(ent + kSpCap);
    int* seg_pre = seg_beg + 2 * kSpRows;
    __shared__ int s_cl[3], s_nn[3];
    __shared__ int whist[kSpThreads / 32][kSpKeys], wpre[kSpThreads / 32][kSpKeys], kstart[kSpKeys + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int o[3] = {(int)blockIdx.x * kSpTX, (int)blockIdx.y * kSpTY, (int)blockIdx.z * kSpTZ};
    const int ext[3] = {min(kSpTX, n - o[0]), min(kSpTY, n - o[1]), min(kSpTZ, n - o[2])};
    const bool alias_z = ext[2] + 3 > n;  // z nodes of one particle may reach the tile twice over the wrap
    for (int i = tid; i < kSpPlaneP * kSpTZ; i += kSpThreads) acc[i] = (T)0;
    if (tid < 3) {
        const double k = (double)nc / (double)n;
        const int od = tid == 0 ? o[0] : tid == 1 ? o[1] : o[2];  // no dynamic indexing (local memory)
        const int ed = tid == 0 ? ext[0] : tid == 1 ? ext[1] : ext[2];
        int lo = (int)floor((double)(od - 2) * k - 1e-9);
        const int hi = (int)floor((double)(od + ed + 1) * k + 1e-9);
        int cnt = hi - lo + 1;
        if (cnt >= nc) {
            lo = 0;
            cnt = nc;
        }
        s_cl[tid] = lo;
        s_nn[tid] = cnt;
    }
    pdl_wait();  // start[] and the particle copies come from the cell-list kernels
    pdl_trigger();
    __syncthreads();
    const int nrows = s_nn[1] * s_nn[2];
    // lane roles in the accumulation: x node kx, y node ky, plane of the warp
    const int kx = lane & 3, ky = (lane >> 2) & 3, pl = 2 * warp + (lane >> 4);
    for (int row0 = 0; row0 < nrows; row0 += kSpRows) {
        const int nr = min(kSpRows, nrows - row0);
        int b0 = 0, l0 = 0, b1 = 0, l1 = 0;
        if (tid < nr) sp_row(start, nc, s_cl, s_nn, row0 + tid, b0, l0, b1, l1);
        int total = 0;
        const int ex0 = sp_block_excl_scan(l0 + l1, &total);  // also orders the previous pass's reads
        if (tid < kSpRows) {
            seg_beg[2 * tid] = b0;
            seg_beg[2 * tid + 1] = b1;
            seg_pre[2 * tid] = ex0;
            seg_pre[2 * tid + 1] = ex0 + l0;
        }
        for (int p0 = 0; p0 < total; p0 += kSpCap) {
            for (int i = tid; i < (kSpThreads / 32) * kSpKeys; i += kSpThreads) (&whist[0][0])[i] = 0;
            __syncthreads();
            // stage 1: one candidate per thread -> tile-local nodes, weights, key
            const int f = p0 + tid;
            int key = -1;
            int loc[3] = {0, 0, 0};
            T w[3][4];
            if (f < total) {
                int lo = 0, hi = 2 * nr - 1;  // last segment starting at or before f
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (seg_pre[mid] <= f) lo = mid;
                    else hi = mid - 1;
                }
                const int s = seg_beg[lo] + (f - seg_pre[lo]);
                int b[3];
                sp_particle(src, s, inv_h, n, b, w);
                bool hit = true;
                int first_z = -1;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    bool any = false;
                    unsigned packed = 0;
#pragma unroll
                    for (int k = 3; k >= 0; --k) {
                        int v = b[d] + k;
                        if (v >= n) v -= n;
                        const int dl = v - o[d];
                        const bool in = (unsigned)dl < (unsigned)ext[d];
                        packed |= (unsigned)(in ? dl : 0xff) << (8 * k);
                        any |= in;
                        if (d == 2 && in) first_z = dl - k;  // the node of weight 0 (may lie below the tile)
                    }
                    loc[d] = (int)packed;
                    hit &= any;
                }
                if (hit) key = alias_z ? 0 : first_z + 3;
            }
            // stable counting sort of this pass's hits by key
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            if (key >= 0 && rank == 0) whist[warp][key] = __popc(peers);
            __syncthreads();
            if (tid < kSpKeys) {
                int run = 0;
#pragma unroll
                for (int ww = 0; ww < kSpThreads / 32; ++ww) {
                    wpre[ww][tid] = run;
                    run += whist[ww][tid];
                }
                whist[0][tid] = run;  // key total (whist is rebuilt next pass)
            }
            __syncthreads();
            if (tid == 0) {
                int run = 0;
                for (int k = 0; k < kSpKeys; ++k) {
                    kstart[k] = run;
                    run += whist[0][k];
                }
                kstart[kSpKeys] = run;
            }
            __syncthreads();
            if (key >= 0) {
                SpEntry<T>& E = ent[kstart[key] + wpre[warp][key] + rank];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    E.loc[d] = loc[d];
#pragma unroll
                    for (int k = 0; k < 4; ++k) E.w[d][k] = w[d][k];
                }
            }
            __syncthreads();
            // stage 2: warp w adds the particles reaching its planes 2w, 2w+1
            // (first z node in [2w-3, 2w+1]) in sorted order
            const int e0 = alias_z ? 0 : kstart[2 * warp];
            const int e1 = alias_z ? kstart[kSpKeys] : kstart[min(2 * warp + 5, kSpKeys)];
            if (2 * warp < ext[2]) {
                for (int e = e0; e < e1; ++e) {
                    const SpEntry<T>& E = ent[e];
                    const int lx = sp_loc(E.loc[0], kx), ly = sp_loc(E.loc[1], ky);
                    const unsigned mz = __vcmpeq4((unsigned)E.loc[2], 0x01010101u * (unsigned)pl);
                    if (lx >= 0 && ly >= 0 && mz != 0u) {
                        const int kz = (__ffs(mz) - 1) >> 3;
                        T* a = acc + pl * kSpPlaneP + ly * kSpRowP + lx;
                        *a += E.w[0][kx] * E.w[1][ky] * E.w[2][kz];
                    }
                }
            }
            __syncthreads();
        }
    }
    // every tile point written once
    if constexpr (VEC) {
        // n % 4 == 0: float4 rows (the tile origin is a multiple of 32)
        for (int i = tid; i < kSpTZ * kSpTY * (kSpTX / 4); i += kSpThreads) {
            const int x4 = i % (kSpTX / 4), ly = (i / (kSpTX / 4)) % kSpTY, lz = i / ((kSpTX / 4) * kSpTY);
            if (4 * x4 >= ext[0] || ly >= ext[1] || lz >= ext[2]) continue;
            const float4 v = *reinterpret_cast<const float4*>(acc + lz * kSpPlaneP + ly * kSpRowP + 4 * x4);
            *reinterpret_cast<float4*>(q + ((int64_t)(o[2] + lz) * n + (o[1] + ly)) * n + o[0] + 4 * x4) = v;
        }
    } else {
        for (int i = tid; i < kSpTZ * kSpTY * kSpTX; i += kSpThreads) {
            const int lx = i % kSpTX, ly = (i / kSpTX) % kSpTY, lz = i / (kSpTX * kSpTY);
            if (lx >= ext[0] || ly >= ext[1] || lz >= ext[2]) continue;
            q[((int64_t)(o[2] + lz) * n + (o[1] + ly)) * n + o[0] + lx] = acc[lz * kSpPlaneP + ly * kSpRowP + lx];
        }
    }
}

inline dim3 spread_grid(int n) {
    return dim3((n + kSpTX - 1) / kSpTX, (n + kSpTY - 1) / kSpTY, (n + kSpTZ - 1) / kSpTZ);
}

// ---------------------------------------------------------------- 3D launch
// Stencil kernels run on a (32, 8) thread block over an (x, y) tile with
// blockIdx.z = z, so no index division is needed.  XDIV = 2 packs two x
// points per thread slot (red-black half sweeps).
#define P3_BX 32
#define P3_BY 8

__device__ __forceinline__ bool xyz3(int n, int& x, int& y, int& z) {
    x = blockIdx.x * P3_BX + threadIdx.x;
    y = blockIdx.y * P3_BY + threadIdx.y;
    z = blockIdx.z;
    return x < n && y < n;
}

// ---------------------------------------------------------------- smoothing
// One explicit diffusion step out = in + c M in (reading of Sec. 2's
// diffusion-based smoothing).  Each thread marches zc planes along z keeping
// the z neighbours in registers (zc planes per thread, a tunable); x and y
// neighbours come through L1.  With
// SUM (the last step) the block also writes the FP64 sum of
// its outputs, from which the neutrality mean is formed.

template <typename T, bool SUM>
__global__ void __launch_bounds__(P3_BX * P3_BY)
k_diffuse(int n, int zc, const T* __restrict__ in, T* __restrict__ out, T c, double* __restrict__ partial) {
    const int x = blockIdx.x * P3_BX + threadIdx.x;
    const int y = blockIdx.y * P3_BY + threadIdx.y;
    const int z0 = blockIdx.z * zc;
    const int z1 = min(z0 + zc, n);
    double acc = 0.0;
    if (x < n && y < n) {
        const int xm = x == 0 ? n - 1 : x - 1, xp = x == n - 1 ? 0 : x + 1;
        const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
        const int plane = n * n;
        const int col = y * n + x;
        T vm = in[(z0 == 0 ? n - 1 : z0 - 1) * plane + col];
        T vc = in[z0 * plane + col];
        for (int z = z0; z < z1; ++z) {
            const int zp = z == n - 1 ? 0 : z + 1;
            const T vp = in[zp * plane + col];
            const int base = z * plane;
            const T sxy = in[base + y * n + xm] + in[base + y * n + xp] + in[base + ym * n + x] + in[base + yp * n + x];
            const T v = vc + c * (sxy + vm + vp - (T)6 * vc);
            out[base + col] = v;
            if (SUM) acc += (double)v;
            vm = vc;
            vc = vp;
        }
    }
    if (SUM) {
        acc = block_sum(acc);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            partial[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = acc;
    }
}

// Compensated FP32 summation for the neutrality block sums: s + c carries a
// running sum with the exact rounding error of every addition (Knuth's
// two-sum), about 48 significant bits after the 32 additions of a thread, at
// FP32 rates; FP64 conversions and adds run at 1/64 of that on this part.
// The pair becomes one FP64 value per thread before the FP64 block sum.
__device__ __forceinline__ void two_sum_add(float& s, float& c, float v) {
    const float t = __fadd_rn(s, v);
    const float bv = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bv)), __fsub_rn(v, bv)));
    s = t;
}

// One explicit diffusion step in FP32 with four x-consecutive points per
// thread (float4 loads and stores; N % 4 == 0).  The x-1 and x+4 neighbours
// of a quad come from the neighbouring lanes by shuffle (the row ends load
// them).  Each thread forms ZC z-consecutive planes; every load of its column
// (planes z0-1 .. z0+ZC), of the y-1 and y+1 rows and of the row-end
// neighbours is issued before the first output is formed, so one L2 round
// trip covers the whole column.  SUM as in k_diffuse.
template <int ZC, bool SUM>
__global__ void __launch_bounds__(P3_BX * P3_BY)
k_diffuse4(int n, const float* __restrict__ in, float* __restrict__ out, float c, double* __restrict__ partial) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x;
    const int q = blockIdx.x * P3_BX + lane;
    const int x = 4 * q;
    const int y = blockIdx.y * P3_BY + threadIdx.y;
    const int z0 = blockIdx.z * ZC;
    const bool live = x < n && y < n;
    const int nq = n >> 2;
    const int yy = live ? y : 0, xx = live ? x : 0;
    const int xl = xx == 0 ? n - 1 : xx - 1;
    const int xr = xx + 4 == n ? 0 : xx + 4;
    const int ym = yy == 0 ? n - 1 : yy - 1, yp = yy == n - 1 ? 0 : yy + 1;
    const int plane = n * n;
    const bool lend = lane == 0 || q - 1 >= nq, rend = lane == P3_BX - 1 || q + 1 >= nq;
    const float4* in4 = reinterpret_cast<const float4*>(in);
    auto wz = [&](int z) { return z < 0 ? z + n : (z >= n ? z - n : z); };
    float4 col[ZC + 2], am[ZC], bp[ZC];
    float lft[ZC], rgt[ZC];
#pragma unroll
    for (int k = 0; k < ZC + 2; ++k) col[k] = in4[(wz(z0 - 1 + k) * plane + yy * n + xx) >> 2];
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const int z = wz(z0 + k);
        am[k] = in4[(z * plane + ym * n + xx) >> 2];
        bp[k] = in4[(z * plane + yp * n + xx) >> 2];
        lft[k] = lend ? in[z * plane + yy * n + xl] : 0.0f;
        rgt[k] = rend ? in[z * plane + yy * n + xr] : 0.0f;
    }
    float acc_s = 0.0f, acc_c = 0.0f;
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const float4 vm = col[k], vc = col[k + 1], vp = col[k + 2], a = am[k], b = bp[k];
        float left = __shfl_up_sync(0xffffffffu, vc.w, 1);
        float right = __shfl_down_sync(0xffffffffu, vc.x, 1);
        if (lend) left = lft[k];
        if (rend) right = rgt[k];
        float4 o;
        o.x = vc.x + c * (left + vc.y + a.x + b.x + vm.x + vp.x - 6.0f * vc.x);
        o.y = vc.y + c * (vc.x + vc.z + a.y + b.y + vm.y + vp.y - 6.0f * vc.y);
        o.z = vc.z + c * (vc.y + vc.w + a.z + b.z + vm.z + vp.z - 6.0f * vc.z);
        o.w = vc.w + c * (vc.z + right + a.w + b.w + vm.w + vp.w - 6.0f * vc.w);
        if (live && z0 + k < n) {
            reinterpret_cast<float4*>(out)[((z0 + k) * plane + yy * n + x) >> 2] = o;
            if (SUM) {
                two_sum_add(acc_s, acc_c, o.x);
                two_sum_add(acc_s, acc_c, o.y);
                two_sum_add(acc_s, acc_c, o.z);
                two_sum_add(acc_s, acc_c, o.w);
            }
        }
    }
    if (SUM) {
        const double acc = block_sum((double)acc_s + (double)acc_c);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            partial[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = acc;
    }
}

// All K diffusion steps of small FP32 meshes in one launch, the mesh resident
// in the (distributed) shared memory of a thread-block cluster.  One cluster
// of cs CTAs per mesh (16 <= n <= 64, n % 4 == 0; cs = cluster_size_for(n),
// the fewest CTAs, 1 to 16, whose slabs fit the shared-memory budget); CTA r
// owns the z planes [r n / cs, (r+1) n / cs) in two shared-memory buffers.  A step
// reads the planes of the current buffer -- the slab's first and last planes'
// outer neighbours from the adjacent CTAs' shared memory (periodic over the
// cluster) -- and writes the next buffer; one cluster barrier separates the
// steps, so every CTA reads only planes the whole cluster has finished.  The
// per-point arithmetic is k_diffuse4's (same operands, same order).  The
// first step reads q from memory, the last writes q^s to memory and to the
// slab.  The neutrality sum is formed per plane (one warp, lanes striding the
// plane with compensated FP32 sums, a fixed butterfly in FP64) and rank 0
// adds the planes in z order, so it does not depend on the cluster size.  The
// launch covers every mesh of a table (one cluster each), so many systems'
// smoothing is one launch.
constexpr int kClMaxCTAs = 16;               // largest cluster (non-portable; opted in per kernel)
constexpr int kClThreads = 512;
constexpr int kClMinN = 16, kClMaxN = 64;
constexpr size_t kClSmemBudget = 200 * 1024;  // both slab buffers of one CTA

struct ClusterMesh {
    const float* q;    // assigned charge, n^3
    float* qs;         // smoothed charge, n^3
    double* qsum;      // FP64 sum of qs (neutrality mean)
    int n, K;
    float c;
    int pad;
};

inline int cluster_planes(int n, int cs) { return (n + cs - 1) / cs; }
inline size_t cluster_smem_bytes(int nmax, int cs) {
    return 2 * sizeof(float) * (size_t)cluster_planes(nmax, cs) * nmax * nmax + 16;
}
inline bool cluster_mesh_ok(int n) { return n >= kClMinN && n <= kClMaxN && n % 4 == 0; }
// CTAs per mesh (a power of two) when `members` meshes share one launch on a
// device of nsm SMs: at least the fewest whose double-buffered slabs fit the
// budget, and then doubled while the launch still has at most one CTA per SM
// (more CTAs per mesh shorten each step; a single mesh gets the largest
// cluster).
inline int cluster_size_for(int n, int members = 1, int nsm = 148) {
    int cs = 1;
    while (cs < kClMaxCTAs && cluster_smem_bytes(n, cs) > kClSmemBudget + 16) cs *= 2;
    while (cs < kClMaxCTAs && 2 * cs * members <= nsm) cs *= 2;
    return cs;
}

static __global__ void __launch_bounds__(kClThreads)
k_diffuse_cluster(const ClusterMesh* __restrict__ tab) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char cl_raw[];
    __shared__ double psum[kClMaxN];  // per local plane
    const int cs = (int)cluster.num_blocks();
    const int member = blockIdx.x / cs;
    const int rank = (int)cluster.block_rank();
    pdl_wait();  // q comes from the assignment kernel
    pdl_trigger();
    const ClusterMesh M = tab[member];
    const int n = M.n, nq = n >> 2, plane = n * n, plane4 = plane >> 2;
    const int z0 = rank * n / cs, z1 = (rank + 1) * n / cs, p = z1 - z0;
    const int pmax = (n + cs - 1) / cs;
    float* const buf0 = reinterpret_cast<float*>(cl_raw);
    float* const buf1 = buf0 + (size_t)pmax * plane;
    const int lo = (rank + cs - 1) % cs, hi = (rank + 1) % cs;  // itself when cs = 1
    const int p_lo = (lo + 1) * n / cs - lo * n / cs;           // planes of the CTA below
    const float4* q4 = reinterpret_cast<const float4*>(M.q) + (size_t)z0 * plane4;
    float4* a4 = reinterpret_cast<float4*>(buf0);
    for (int i = threadIdx.x; i < p * plane4; i += kClThreads) a4[i] = q4[i];
    cluster.sync();
    const float c = M.c;
    // work items: an x-quad column (qx, y) over a run of L consecutive local
    // planes, marched in z with the lower and centre planes in registers;
    // L is chosen so the items cover the block about once
    const int ncol = plane4;
    const int L = max(1, min(p, (p * ncol + kClThreads - 1) / kClThreads));
    const int nrun = (p + L - 1) / L;
    for (int st = 0; st < M.K; ++st) {
        const float* A = (st & 1) ? buf1 : buf0;
        float* B = (st & 1) ? buf0 : buf1;
        const float* Alo = cluster.map_shared_rank(const_cast<float*>(A), lo) + (size_t)(p_lo - 1) * plane;
        const float* Ahi = cluster.map_shared_rank(const_cast<float*>(A), hi);
        const bool last = st == M.K - 1;
        for (int it = threadIdx.x; it < ncol * nrun; it += kClThreads) {
            const int run = it / ncol, col = it - run * ncol, y = col / nq, qx = col - y * nq, x = 4 * qx;
            const int za = run * L, zb = min(p, za + L);
            const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
            const int xl = x == 0 ? n - 1 : x - 1, xr = x + 4 == n ? 0 : x + 4;
            const int off = y * n + x;
            float4 vm = *reinterpret_cast<const float4*>((za > 0 ? A + (size_t)(za - 1) * plane : Alo) + off);
            float4 vc = *reinterpret_cast<const float4*>(A + (size_t)za * plane + off);
            for (int zl = za; zl < zb; ++zl) {
                const float* Ap = A + (size_t)zl * plane;
                const float4 vp = *reinterpret_cast<const float4*>((zl < p - 1 ? Ap + plane : Ahi) + off);
                const float4 a = *reinterpret_cast<const float4*>(Ap + ym * n + x);
                const float4 b = *reinterpret_cast<const float4*>(Ap + yp * n + x);
                const float left = Ap[y * n + xl];
                const float right = Ap[y * n + xr];
                float4 o;
                o.x = vc.x + c * (left + vc.y + a.x + b.x + vm.x + vp.x - 6.0f * vc.x);
                o.y = vc.y + c * (vc.x + vc.z + a.y + b.y + vm.y + vp.y - 6.0f * vc.y);
                o.z = vc.z + c * (vc.y + vc.w + a.z + b.z + vm.z + vp.z - 6.0f * vc.z);
                o.w = vc.w + c * (vc.z + right + a.w + b.w + vm.w + vp.w - 6.0f * vc.w);
                const size_t io = (size_t)zl * plane4 + col;
                if (last) reinterpret_cast<float4*>(M.qs)[(size_t)z0 * plane4 + io] = o;
                reinterpret_cast<float4*>(B)[io] = o;
                vm = vc;
                vc = vp;
            }
        }
        cluster.sync();  // B complete everywhere before anyone reads it; A free
    }
    // the last step's output is in buffer K & 1 (K >= 1; K = 0 leaves q itself)
    const float* Q = M.K == 0 ? buf0 : ((M.K & 1) ? buf1 : buf0);
    if (M.K == 0) {
        for (int i = threadIdx.x; i < p * plane4; i += kClThreads)
            reinterpret_cast<float4*>(M.qs)[(size_t)z0 * plane4 + i] = a4[i];
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int zl = warp; zl < p; zl += kClThreads / 32) {
        const float* Qp = Q + (size_t)zl * plane;
        float s = 0.0f, e = 0.0f;
        for (int j = lane; j < plane; j += 32) two_sum_add(s, e, Qp[j]);
        double v = (double)s + (double)e;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) psum[zl] = v;
    }
    cluster.sync();
    if (rank == 0 && threadIdx.x == 0) {
        double tot = 0.0;  // planes in z order: r ascending, then its planes
        for (int r = 0; r < cs; ++r) {
            const double* ps = cluster.map_shared_rank(psum, r);
            const int pr = (r + 1) * n / cs - r * n / cs;
            for (int zl = 0; zl < pr; ++zl) tot += ps[zl];
        }
        M.qsum[0] = tot;
    }
    cluster.sync();  // the other CTAs' psum stays alive until rank 0 has read it
}

// Two explicit diffusion steps in one pass: (I + cM)^2 written out as one
// 25-point stencil,
//   (I + cM)^2 = (1 - 12c + 42c^2) I + (2c - 12c^2) S1 + c^2 S2 + 2c^2 D,
// S1 the 6 nearest neighbours, S2 the 6 axial neighbours at distance 2, D the
// 12 face diagonals (M^2 = 42 I - 12 S1 + S2 + 2 D for the 7-point M).  The
// same linear operator as two launches of k_diffuse4, with one pass over
// memory.  FP32, four x points per thread (N % 4 == 0), ZC planes per
// thread with every load issued up front; x neighbours up to distance 2 by
// shuffles (row ends load them).  SUM as in k_diffuse.
template <int ZC, bool SUM>
__global__ void __launch_bounds__(P3_BX * P3_BY)
k_diffuse4x2(int n, const float* __restrict__ in, float* __restrict__ out, float a0, float a1, float a2, float a3,
             double* __restrict__ partial) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x;
    const int q = blockIdx.x * P3_BX + lane;
    const int x = 4 * q;
    const int y = blockIdx.y * P3_BY + threadIdx.y;
    const int z0 = blockIdx.z * ZC;
    const bool live = x < n && y < n;
    const int nq = n >> 2;
    const int yy = live ? y : 0, xx = live ? x : 0;
    auto wr = [n](int v) { return v < 0 ? v + n : (v >= n ? v - n : v); };
    const int xl1 = wr(xx - 1), xl2 = wr(xx - 2), xr1 = wr(xx + 4), xr2 = wr(xx + 5);
    const int ym1 = wr(yy - 1), yp1 = wr(yy + 1), ym2 = wr(yy - 2), yp2 = wr(yy + 2);
    const int plane = n * n;
    const bool lend = lane == 0 || q - 1 >= nq, rend = lane == P3_BX - 1 || q + 1 >= nq;
    const float4* in4 = reinterpret_cast<const float4*>(in);
    auto ld4 = [&](int z, int row) { return in4[(wr(z) * plane + row * n + xx) >> 2]; };
    auto ld1 = [&](int z, int row, int xi) { return in[wr(z) * plane + row * n + xi]; };
    float4 col[ZC + 4], rm[ZC + 2], rp[ZC + 2], rm2[ZC], rp2[ZC];
    float cl2[ZC], cr2[ZC], ml1[ZC], mr1[ZC], pl1[ZC], pr1[ZC], zl1[ZC + 2], zr1[ZC + 2];
#pragma unroll
    for (int k = 0; k < ZC + 4; ++k) col[k] = ld4(z0 - 2 + k, yy);             // (y, z0-2+k)
#pragma unroll
    for (int k = 0; k < ZC + 2; ++k) {
        rm[k] = ld4(z0 - 1 + k, ym1);                                          // (y-1, z0-1+k)
        rp[k] = ld4(z0 - 1 + k, yp1);                                          // (y+1, z0-1+k)
        zl1[k] = lend ? ld1(z0 - 1 + k, yy, xl1) : 0.0f;                       // (x-1, y, z0-1+k)
        zr1[k] = rend ? ld1(z0 - 1 + k, yy, xr1) : 0.0f;                       // (x+4, y, z0-1+k)
    }
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        rm2[k] = ld4(z0 + k, ym2);
        rp2[k] = ld4(z0 + k, yp2);
        cl2[k] = lend ? ld1(z0 + k, yy, xl2) : 0.0f;
        cr2[k] = rend ? ld1(z0 + k, yy, xr2) : 0.0f;
        ml1[k] = lend ? ld1(z0 + k, ym1, xl1) : 0.0f;
        mr1[k] = rend ? ld1(z0 + k, ym1, xr1) : 0.0f;
        pl1[k] = lend ? ld1(z0 + k, yp1, xl1) : 0.0f;
        pr1[k] = rend ? ld1(z0 + k, yp1, xr1) : 0.0f;
    }
    // x neighbours at distance 1 (and 2 for the centre row) of a row quad
    auto xn1 = [&](const float4& v, float lend_v, float rend_v, float& l1, float& r1) {
        l1 = __shfl_up_sync(0xffffffffu, v.w, 1);
        r1 = __shfl_down_sync(0xffffffffu, v.x, 1);
        if (lend) l1 = lend_v;
        if (rend) r1 = rend_v;
    };
    float acc_s = 0.0f, acc_c = 0.0f;
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const float4 c = col[k + 2], czm = col[k + 1], czp = col[k + 3], czm2 = col[k], czp2 = col[k + 4];
        const float4 ym = rm[k + 1], yp = rp[k + 1];
        float cl1, cr1, yml1, ymr1, ypl1, ypr1, zml1, zmr1, zpl1, zpr1;
        xn1(c, zl1[k + 1], zr1[k + 1], cl1, cr1);
        float cl2v = __shfl_up_sync(0xffffffffu, c.z, 1), cr2v = __shfl_down_sync(0xffffffffu, c.y, 1);
        if (lend) cl2v = cl2[k];
        if (rend) cr2v = cr2[k];
        xn1(ym, ml1[k], mr1[k], yml1, ymr1);
        xn1(yp, pl1[k], pr1[k], ypl1, ypr1);
        xn1(czm, zl1[k], zr1[k], zml1, zmr1);
        xn1(czp, zl1[k + 2], zr1[k + 2], zpl1, zpr1);
        const float C8[8] = {cl2v, cl1, c.x, c.y, c.z, c.w, cr1, cr2v};
        const float YM[6] = {yml1, ym.x, ym.y, ym.z, ym.w, ymr1};
        const float YP[6] = {ypl1, yp.x, yp.y, yp.z, yp.w, ypr1};
        const float ZM[6] = {zml1, czm.x, czm.y, czm.z, czm.w, zmr1};
        const float ZP[6] = {zpl1, czp.x, czp.y, czp.z, czp.w, zpr1};
        const float YMZM[4] = {rm[k].x, rm[k].y, rm[k].z, rm[k].w}, YMZP[4] = {rm[k + 2].x, rm[k + 2].y, rm[k + 2].z, rm[k + 2].w};
        const float YPZM[4] = {rp[k].x, rp[k].y, rp[k].z, rp[k].w}, YPZP[4] = {rp[k + 2].x, rp[k + 2].y, rp[k + 2].z, rp[k + 2].w};
        const float YM2[4] = {rm2[k].x, rm2[k].y, rm2[k].z, rm2[k].w}, YP2[4] = {rp2[k].x, rp2[k].y, rp2[k].z, rp2[k].w};
        const float ZM2[4] = {czm2.x, czm2.y, czm2.z, czm2.w}, ZP2[4] = {czp2.x, czp2.y, czp2.z, czp2.w};
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float s1 = C8[j + 1] + C8[j + 3] + YM[j + 1] + YP[j + 1] + ZM[j + 1] + ZP[j + 1];
            const float s2 = C8[j] + C8[j + 4] + YM2[j] + YP2[j] + ZM2[j] + ZP2[j];
            const float d = YM[j] + YM[j + 2] + YP[j] + YP[j + 2] + ZM[j] + ZM[j + 2] + ZP[j] + ZP[j + 2] +
                            YMZM[j] + YMZP[j] + YPZM[j] + YPZP[j];
            o[j] = a0 * C8[j + 2] + a1 * s1 + a2 * s2 + a3 * d;
        }
        if (live && z0 + k < n) {
            reinterpret_cast<float4*>(out)[((z0 + k) * plane + yy * n + x) >> 2] = make_float4(o[0], o[1], o[2], o[3]);
            if (SUM) {
#pragma unroll
                for (int j = 0; j < 4; ++j) two_sum_add(acc_s, acc_c, o[j]);
            }
        }
    }
    if (SUM) {
        const double acc = block_sum((double)acc_s + (double)acc_c);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            partial[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = acc;
    }
}

// S explicit diffusion steps fused in one launch (2.5D temporal blocking).
// A block owns an output tile of TX x TY columns and zc planes; its
// (TX + 2S) x (TY + 2S) threads each hold one column of the haloed tile and
// stream z from z0 - S to z0 + zc + S.  When input plane z_in arrives, level
// t (t diffusion steps applied) is formed at plane z_in - t from level t - 1:
// its z neighbours come from the thread's register window, its x and y
// neighbours from the plane of level t - 1 published to shared memory one
// z-step earlier (double buffered, one barrier per z-step).  Level t is valid
// on the tile shrunk by t on each side, so the interior receives S exact
// steps; periodic wrap is applied to every loaded index.  SUM adds the FP64
// block sum of the outputs (neutrality mean) as in k_diffuse.
template <typename T, int S, int TX, int TY, bool SUM>
__global__ void __launch_bounds__((TX + 2 * S) * (TY + 2 * S))
k_diffuse_tb(int n, int zc, const T* __restrict__ in, T* __restrict__ out, T c, double* __restrict__ partial) {
    constexpr int WX = TX + 2 * S, WY = TY + 2 * S, W = WX * WY;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* sm = reinterpret_cast<T*>(sm_raw);  // [2 parities][S levels][W]
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * WX + tx;
    const int gx = (int)blockIdx.x * TX + tx - S;
    const int gy = (int)blockIdx.y * TY + ty - S;
    const int x = ((gx % n) + n) % n, y = ((gy % n) + n) % n;
    const int col = y * n + x, plane = n * n;
    const int z0 = blockIdx.z * zc;
    const int zend = min(z0 + zc, n);
    const bool writer = tx >= S && tx < S + TX && ty >= S && ty < S + TY && gx < n && gy < n;
    T win[S][3];
#pragma unroll
    for (int t = 0; t < S; ++t) win[t][0] = win[t][1] = win[t][2] = (T)0;
    double acc = 0.0;
    const int zstart = z0 - S;
    const int nsteps = (zend - z0) + 2 * S;
    // input planes are fetched two z-steps ahead so their latency overlaps
    // the current step's work and barrier
    auto fetch = [&](int zi) -> T {
        int zw = zi % n;
        if (zw < 0) zw += n;
        return in[zw * plane + col];
    };
    T pf0 = fetch(zstart), pf1 = fetch(zstart + 1);
    for (int st = 0; st < nsteps; ++st) {
        const int zin = zstart + st;
        const int cur = st & 1, prev = cur ^ 1;
        const T v0 = pf0;
        pf0 = pf1;
        if (st + 2 < nsteps) pf1 = fetch(zin + 2);
        win[0][0] = win[0][1];
        win[0][1] = win[0][2];
        win[0][2] = v0;
        sm[(cur * S + 0) * W + tid] = v0;
#pragma unroll
        for (int t = 1; t <= S; ++t) {
            T vt = (T)0;
            if (tx >= t && tx < WX - t && ty >= t && ty < WY - t) {
                const T* pl = sm + (prev * S + (t - 1)) * W;
                const T mid = win[t - 1][1];
                const T sxy = pl[tid - 1] + pl[tid + 1] + pl[tid - WX] + pl[tid + WX];
                vt = mid + c * (sxy + win[t - 1][0] + win[t - 1][2] - (T)6 * mid);
            }
            if (t < S) {
                win[t][0] = win[t][1];
                win[t][1] = win[t][2];
                win[t][2] = vt;
                sm[(cur * S + t) * W + tid] = vt;
            } else {
                const int zo = zin - S;
                if (writer && zo >= z0 && zo < zend) {
                    out[zo * plane + col] = vt;
                    if (SUM) acc += (double)vt;
                }
            }
        }
        __syncthreads();
    }
    if (SUM) {
        acc = block_sum(acc);
        if (tid == 0) partial[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = acc;
    }
}

// S explicit diffusion steps per pass over memory in FP32 quads (N % 4 ==
// 0), 2.5D temporal blocking with asynchronous copies.  A block of 256
// threads holds a haloed tile of 64 x 32 columns (16 quads x 32 rows; one
// quad of halo on each x side, S rows on each y side); thread (q, p) owns the
// quad q of rows 2p and 2p+1.  The block streams z from z0 - S to
// z0 + zc + S.  The input planes of the tile arrive through a ring of
// kTqRing shared-memory planes filled by cp.async 16-byte copies issued
// kTqAhead planes ahead (no registers held by loads in flight).  When input
// plane z_in is resident, level t (t steps applied) is formed at plane
// z_in - t: each thread keeps, for both of its rows, a register window of
// three consecutive planes of the input and of every level below S (the z
// neighbours); the y neighbour between its two rows is in registers, the
// outer two come from the plane published in shared memory one z step
// earlier (the input ring for level 1; double-buffered level planes above);
// x neighbours of a quad come from the adjacent lanes.  Values outside the
// region where level t is exact (t points in from the haloed tile's edge)
// are formed but never reach an output.  The per-point arithmetic is
// k_diffuse4's (same operands, same order), so S launches of k_diffuse4 and
// one of this kernel give the same bits.  SUM as in k_diffuse4.
constexpr int kTq = 16, kTh = 32, kTqThreads = kTq * kTh / 2;  // quads per row, rows, threads
constexpr int kTqAhead = 5, kTqRing = kTqAhead + 3;            // planes in flight; ring planes
constexpr int kTqTX = 4 * kTq - 8;                             // output columns per tile (56)
template <int S>
constexpr int tq_tile_y() { return kTh - 2 * S; }
template <int S>
constexpr size_t tq_smem_bytes() {
    return sizeof(float4) * kTq * kTh * (kTqRing + 2 * (S - 1));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One diffusion step of a quad (k_diffuse4's expression); the x neighbours
// outside the quad come from the lanes on either side.
__device__ __forceinline__ float4 diffuse_quad(float4 vc, float4 vm, float4 vp, float4 a, float4 b, float c) {
    const float left = __shfl_up_sync(0xffffffffu, vc.w, 1);
    const float right = __shfl_down_sync(0xffffffffu, vc.x, 1);
    float4 o;
    o.x = vc.x + c * (left + vc.y + a.x + b.x + vm.x + vp.x - 6.0f * vc.x);
    o.y = vc.y + c * (vc.x + vc.z + a.y + b.y + vm.y + vp.y - 6.0f * vc.y);
    o.z = vc.z + c * (vc.y + vc.w + a.z + b.z + vm.z + vp.z - 6.0f * vc.z);
    o.w = vc.w + c * (vc.z + right + a.w + b.w + vm.w + vp.w - 6.0f * vc.w);
    return o;
}

template <int S, bool SUM>
__global__ void __launch_bounds__(kTqThreads, 2)
k_diffuse_tq(int n, int zc, const float* __restrict__ in, float* __restrict__ out, float c,
             double* __restrict__ partial) {
    constexpr int TY = tq_tile_y<S>();
    constexpr int PL = kTq * kTh;  // float4 per plane
    constexpr int NW = S > 1 ? S - 1 : 1;
    extern __shared__ __align__(16) unsigned char tq_raw[];
    float4* ring = reinterpret_cast<float4*>(tq_raw);  // [kTqRing][kTh][kTq]
    float4* lvl = ring + kTqRing * PL;                 // [S-1][2][kTh][kTq]
    const int tid = threadIdx.x, q = tid & (kTq - 1), r0 = 2 * (tid / kTq), r1 = r0 + 1;
    const int x0 = blockIdx.x * kTqTX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * zc, zend = min(z0 + zc, n);
    const size_t plane = (size_t)n * n;
    int gx = (x0 - 4 + 4 * q) % n, gy0 = (y0 - S + r0) % n, gy1 = (y0 - S + r1) % n;  // the quads this thread copies
    gx = gx < 0 ? gx + n : gx;
    gy0 = gy0 < 0 ? gy0 + n : gy0;
    gy1 = gy1 < 0 ? gy1 + n : gy1;
    const size_t col0 = (size_t)gy0 * n + gx, col1 = (size_t)gy1 * n + gx;
    const int zstart = z0 - S, nsteps = (zend - z0) + 2 * S;
    pdl_wait();  // `in` comes from the previous launch
    pdl_trigger();
    auto issue = [&](int st) {  // input plane zstart + st into ring slot st % kTqRing
        if (st < nsteps) {
            int z = (zstart + st) % n;
            z = z < 0 ? z + n : z;
            float4* d = ring + (st % kTqRing) * PL + q;
            cp_async16(d + r0 * kTq, in + (size_t)z * plane + col0);
            cp_async16(d + r1 * kTq, in + (size_t)z * plane + col1);
        }
        cp_async_commit();  // one group per plane, empty past the end
    };
#pragma unroll
    for (int d = 0; d < kTqAhead; ++d) issue(d);
    const int ra = r0 == 0 ? 0 : r0 - 1, rb = r1 == kTh - 1 ? r1 : r1 + 1;  // outer y neighbours (edge rows are halo)
    const bool wq = q >= 1 && q < kTq - 1 && x0 + 4 * (q - 1) < n;
    const bool w0 = wq && r0 >= S && r0 < kTh - S && y0 + r0 - S < n;
    const bool w1 = wq && r1 >= S && r1 < kTh - S && y0 + r1 - S < n;
    const size_t oc0 = (size_t)(y0 + r0 - S) * n + x0 + 4 * (q - 1), oc1 = oc0 + n;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 i0[3] = {z4, z4, z4}, i1[3] = {z4, z4, z4};  // input window, rows r0 and r1
    float4 w[NW][2][3];                                 // level windows
#pragma unroll
    for (int t = 0; t < NW; ++t)
#pragma unroll
        for (int k = 0; k < 3; ++k) w[t][0][k] = w[t][1][k] = z4;
    float acc_s = 0.0f, acc_c = 0.0f;
#pragma unroll 3  // the three-plane windows rotate by renaming
    for (int st = 0; st < nsteps; ++st) {
        cp_async_wait<kTqAhead - 1>();  // this thread's copies of plane st have landed
        __syncthreads();                // everyone's, and the previous step's reads are done
        issue(st + kTqAhead);           // into the slot of plane st - 3, no longer read
        const int cur = st & 1, prv = cur ^ 1;
        const float4* Pn = ring + (st % kTqRing) * PL;                   // plane st
        const float4* Pc = ring + ((st + kTqRing - 1) % kTqRing) * PL;  // plane st - 1
        i0[0] = i0[1];
        i0[1] = i0[2];
        i0[2] = Pn[r0 * kTq + q];
        i1[0] = i1[1];
        i1[1] = i1[2];
        i1[2] = Pn[r1 * kTq + q];
        // level 1 at input plane st - 1
        float4 o0 = diffuse_quad(i0[1], i0[0], i0[2], Pc[ra * kTq + q], i1[1], c);
        float4 o1 = diffuse_quad(i1[1], i1[0], i1[2], i0[1], Pc[rb * kTq + q], c);
#pragma unroll
        for (int t = 2; t <= S; ++t) {
            // publish level t - 1 (formed at plane st - (t - 1)) and form level t from it
            float4* W0 = w[t - 2][0];
            float4* W1 = w[t - 2][1];
            W0[0] = W0[1];
            W0[1] = W0[2];
            W0[2] = o0;
            W1[0] = W1[1];
            W1[1] = W1[2];
            W1[2] = o1;
            float4* Lc = lvl + ((t - 2) * 2 + cur) * PL;
            Lc[r0 * kTq + q] = o0;
            Lc[r1 * kTq + q] = o1;
            const float4* L = lvl + ((t - 2) * 2 + prv) * PL;
            o0 = diffuse_quad(W0[1], W0[0], W0[2], L[ra * kTq + q], W1[1], c);
            o1 = diffuse_quad(W1[1], W1[0], W1[2], W0[1], L[rb * kTq + q], c);
        }
        // o0, o1: level S at plane st - S (input numbering), output plane zstart + st - S
        const int zo = zstart + st - S;
        if (zo >= z0 && zo < zend) {
            float* op = out + (size_t)zo * plane;
            if (w0) {
                *reinterpret_cast<float4*>(op + oc0) = o0;
                if (SUM) {
                    two_sum_add(acc_s, acc_c, o0.x);
                    two_sum_add(acc_s, acc_c, o0.y);
                    two_sum_add(acc_s, acc_c, o0.z);
                    two_sum_add(acc_s, acc_c, o0.w);
                }
            }
            if (w1) {
                *reinterpret_cast<float4*>(op + oc1) = o1;
                if (SUM) {
                    two_sum_add(acc_s, acc_c, o1.x);
                    two_sum_add(acc_s, acc_c, o1.y);
                    two_sum_add(acc_s, acc_c, o1.z);
                    two_sum_add(acc_s, acc_c, o1.w);
                }
            }
        }
    }
    cp_async_wait<0>();
    if (SUM) {
        const double acc = block_sum((double)acc_s + (double)acc_c);
        if (tid == 0) partial[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = acc;
    }
}

// ---------------------------------------------------------------- reductions
template <typename T>
__global__ void k_sum_partial(int64_t m, const T* __restrict__ x, double* __restrict__ partial) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)x[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

template <typename T>
__global__ void k_dot_partial(int64_t m, const double* __restrict__ a, const T* __restrict__ b,
                              double* __restrict__ partial) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        acc += a[i] * (double)b[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// Kinetic-energy partials: sum m v^2 over particles.
static __global__ void k_mv2_partial(int np, const double* __restrict__ v, const double* __restrict__ m,
                              double* __restrict__ partial) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x)
        acc += m[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// Sum of nb partials (in a fixed order) into out[0].
static __global__ void k_sum_final(int nb, const double* __restrict__ partial, double* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) out[0] = acc;
}

// ---------------------------------------------------------------- gauge mode
// M annihilates constants, so the correction y (z in fixed point) of a solve
// is defined up to a constant, and so is the potential (reading A5: keep
// mean(y) = 0).  The multiplier predictor extrapolates the history -- order
// 3 is a triple integrator of whatever constant the V-cycles leave behind --
// so a constant that is not removed grows with the step count until it
// swamps the precision of phi.  Each history buffer therefore carries its
// own sum in one extra slot, and the predictor removes the mean of its
// guess: a constant shift of the guess leaves every residual and every force
// unchanged.  FP64: the field-update kernel measures the sum of y* (its
// rounding does not propagate, the next step measures again).  Mixed: the
// sum of z in fixed point is kept exactly in 64-bit integers -- the
// prediction records the guess's exact remainder after removing an integer
// mean, each residual update adds its increments' exact sum -- so the
// recorded sums equal the buffers' sums bit for bit.
//
// Block sums of v, reduced to *out by the block that finishes last (fixed
// order over the partials, so the sum is the same on every run).
__device__ __forceinline__ void sum_last_block(double v, double* __restrict__ partial, unsigned* __restrict__ arrive,
                                               double* __restrict__ out) {
    __shared__ int last_s;
    const double bs = block_sum(v);
    const int nb = gridDim.x;
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = bs;
        __threadfence();
        last_s = atomicAdd(arrive, 1u) == (unsigned)(nb - 1);
    }
    __syncthreads();
    if (!last_s) return;
    __threadfence();
    double a = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) a += __ldcg(partial + i);
    a = block_sum(a);
    if (threadIdx.x == 0) {
        *arrive = 0u;
        *out = a;
    }
}

// Mean of the order-`order` guess from the sums of the history buffers
// (slot m of each), per point.
__device__ __forceinline__ double guess_mean(int order, const double* __restrict__ y1, const double* __restrict__ y2,
                                             const double* __restrict__ y3, int64_t m) {
    if (order == 1) return y1[m] / (double)m;
    if (order == 2) return (2.0 * y1[m] - y2[m]) / (double)m;
    if (order == 3) return (3.0 * y1[m] - 3.0 * y2[m] + y3[m]) / (double)m;
    return 0.0;
}

// ---------------------------------------------------------------- Mass-Zero
// psi = (h/4pi) M phi is carried from step to step (it follows from the final
// FP64 residual: (h/4pi) M phi^{k+1} = sigma_p - M y* - q^s), so the
// prediction needs no stencil:
//   sigma_p = (h/4pi) M (2 phi^k - phi^{k-1}) + q^s - mean      (Eq. 17)
//           = 2 psi^k - psi^{k-1} + q^s - mean(q^s)
// and the multiplier guess y0 (Sec. 3.3): order 0 -> 0, 1 -> y^k,
// 2 -> 2y^k - y^{k-1}, 3 -> 3y^k - 3y^{k-1} + y^{k-2}, its mean removed.
template <typename T>
__global__ void __launch_bounds__(P3_THREADS)
k_predict(int64_t m, const double* __restrict__ psik, const double* __restrict__ psikm1,
          const T* __restrict__ qs, const double* __restrict__ qsum, double inv_pts,
          const double* __restrict__ y1, const double* __restrict__ y2, const double* __restrict__ y3,
          int order, double* __restrict__ sig, double* __restrict__ y0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const double mean = qsum[0] * inv_pts;
    sig[i] = 2.0 * psik[i] - psikm1[i] + ((double)qs[i] - mean);
    double g = 0.0;
    if (order == 1) g = y1[i];
    else if (order == 2) g = 2.0 * y1[i] - y2[i];
    else if (order == 3) g = 3.0 * y1[i] - 3.0 * y2[i] + y3[i];
    y0[i] = g - guess_mean(order, y1, y2, y3, m);  // the gauge mode removed
}

// Fine-level FP64 residual r = sigma_p - M y (Eq. 20's argument): kept in
// FP64 (rfin, for the psi update) and in the bulk type (input of the
// correction V-cycle).  Each block walks z planes blockIdx.z, +gridDim.z, ...
// and writes max |r| over its points to bmax (NaN or Inf recorded as +Inf);
// the check kernel reduces those block maxima.
template <typename T>
__global__ void __launch_bounds__(P3_BX * P3_BY)
k_resid_fine(int n, const double* __restrict__ yv, const double* __restrict__ sig, T* __restrict__ r,
             double* __restrict__ rfin, double* __restrict__ bmax) {
    const int x = blockIdx.x * P3_BX + threadIdx.x;
    const int y = blockIdx.y * P3_BY + threadIdx.y;
    float a = 0.0f;
    if (x < n && y < n) {
        for (int z = blockIdx.z; z < n; z += gridDim.z) {
            const int i = (z * n + y) * n + x;
            const double res = sig[i] - (nb6(yv, x, y, z, n) - 6.0 * yv[i]);
            r[i] = (T)res;
            rfin[i] = res;
            // the max-norm is taken on the FP32-rounded |r| (relative error
            // 6e-8, far inside any tolerance); NaN becomes +Inf
            const float v = fabsf((float)res);
            a = (v == v) ? fmaxf(a, v) : __int_as_float(0x7f800000);
        }
    }
    const double am = block_max((double)a);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        bmax[(blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = am;
}

// y += e (FP64 accumulation of the correction).
template <typename T>
__global__ void k_add_correction(int64_t m, double* __restrict__ yv, const T* __restrict__ e) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) yv[i] += (double)e[i];
}

// Field update (supporting information Sec. 1), written over the k-1 slots:
//   phi^{k+1} = 2 phi^k - phi^{k-1} - (4pi/h) y*
//   psi^{k+1} = (h/4pi) M phi^{k+1} = r_final - (q^s - mean)
// Grid-stride over the points; the sum of y* goes to yv[m] (gauge mode).
template <typename T>
__global__ void __launch_bounds__(P3_THREADS)
k_update(int64_t m, const double* __restrict__ phik, double* __restrict__ phikm1,
         double* __restrict__ psikm1, double* __restrict__ yv,
         const double* __restrict__ rfin, const T* __restrict__ qs,
         const double* __restrict__ qsum, double inv_pts, double coef, float* __restrict__ phi32,
         double* __restrict__ partial, unsigned* __restrict__ arrive) {
    double ys = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const double y = yv[i];
        ys += y;
        const double p = 2.0 * phik[i] - phikm1[i] - coef * y;
        phikm1[i] = p;
        psikm1[i] = rfin[i] - ((double)qs[i] - qsum[0] * inv_pts);
        // FP32 copy for the mixed-precision interpolation, relative to one node
        // value of phi^k so the constant mode of phi (a gauge freedom) never eats
        // FP32 digits; the central differences are unchanged by it
        if (phi32 != nullptr) phi32[i] = (float)(p - phik[0]);
    }
    sum_last_block(ys, partial, arrive, yv + m);
}

// ---------------------------------------------------------------- fixed point
// Mixed precision carries the constraint algebra of Eqs. 16-17 and 20 in
// 64-bit fixed point, value x 2^40 in potential units (e/A; resolution
// 9.1e-13, range +-8.4e6): the potential phi, Psi = M phi, the correction
// z = (4pi/h) y, the predicted residual s = M phi_p + (4pi/h)(q^s - mean)
// = (4pi/h) sigma_p and the residual r = s - M z.  Sums, differences and the
// integer 7-point stencil are exact in this form, so Psi^{k+1} = M phi^{k+1}
// holds bit for bit at every step and is carried forward instead of
// recomputed; FP32 values enter once each (the smoothed charge, the V-cycle
// corrections) and are accounted for exactly in both phi and Psi.  The
// constant mode of phi (a gauge freedom) may wrap around in two's
// complement: every use takes differences of phi values, which stay exact.
typedef long long fix_t;
constexpr float kFixOne = 1099511627776.0f;        // 2^40
constexpr float kFixInv = 1.0f / 1099511627776.0f;  // 2^-40, exact

// int64 -> float as hi 2^32 + lo with 32-bit conversions (round-off of one
// or two float ulps; used for V-cycle inputs and the max-norm only).
__device__ __forceinline__ float fix_to_float(fix_t v) {
    const int hi = (int)(v >> 32);
    const unsigned lo = (unsigned)(v & 0xffffffffll);
    return fmaf((float)hi, 4294967296.0f, (float)lo) * kFixInv;
}

// float -> nearest-or-truncated fixed point with 32-bit conversions.  Small
// values convert directly; large ones (|f| >= 2^31, so f is a multiple of
// 2^8) split exactly into 2^32 hi + lo.  Which integer is chosen does not
// matter for exactness: the same integer enters phi and Psi.  Finite inputs
// of magnitude below 2^23 only (the callers flag non-finite values).
// (Measured and not kept: one direct float-to-int64 conversion, which gives
// the same integers, took the residual update at 128^3 from 28.5 to 39 us.)
__device__ __forceinline__ fix_t float_to_fix(float e) {
    const float f = e * kFixOne;
    if (fabsf(f) < 2147483648.0f) return (fix_t)__float2int_rn(f);
    const float hi = truncf(f * (1.0f / 4294967296.0f));
    const float lo = fmaf(-hi, 4294967296.0f, f);  // exact: multiple of 2^8, |lo| < 2^32
    return (fix_t)__float2int_rz(hi) * 4294967296ll + 2ll * (fix_t)__float2int_rn(0.5f * lo);
}

// (4pi/h)(q^s - mean) in fixed point, rounded the same way wherever it is
// formed (no contraction into an FMA).
__device__ __forceinline__ fix_t charge_term(float qs, float mean, float u) {
    return float_to_fix(__fmul_rn(__fsub_rn(qs, mean), u));
}

// Field update in fixed point, written over the k-1 slots:
//   phi^{k+1} = 2 phi^k - phi^{k-1} - z*
//   Psi^{k+1} = M phi^{k+1} = r_final - (4pi/h)(q^s - mean)
// and the FP32 copy of phi^{k+1} - phi^k[0] for the interpolation.
// (The sum of z*, slot m of z's buffer, is kept by the prediction and the
// residual updates: see k_predict_resid_fix and k_resid_update_fix.)
static __global__ void __launch_bounds__(P3_THREADS)
k_update_fix(int64_t m, const fix_t* __restrict__ phik, fix_t* __restrict__ phikm1, fix_t* __restrict__ Psikm1,
             const fix_t* __restrict__ z, const fix_t* __restrict__ rfin, const float* __restrict__ qs,
             const double* __restrict__ qsum, double inv_pts, float u, float* __restrict__ phi32) {
    __shared__ float mean_s;
    __shared__ fix_t ref_s;
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0) {
        mean_s = (float)(qsum[0] * inv_pts);
        ref_s = phik[0];
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const fix_t p = 2 * phik[i] - phikm1[i] - z[i];
    phikm1[i] = p;
    Psikm1[i] = rfin[i] - charge_term(qs[i], mean_s, u);
    phi32[i] = fix_to_float(p - ref_s);
}

// Partial sums of (phi_i - phi_0) b_i with phi in fixed point (energy
// 1/2 phi^T q; the reference value removes the gauge constant).
template <typename T>
__global__ void k_dot_partial_fix(int64_t m, const fix_t* __restrict__ a, const T* __restrict__ b,
                                  double* __restrict__ partial) {
    const fix_t ref = a[0];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        acc += (double)(a[i] - ref) * (double)b[i];
    acc = block_sum(acc) * (1.0 / 1099511627776.0);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// Convergence control of the correction solve (Eq. 20), one block: reduces
// the block maxima of the residual just computed to max|r| and decides whether another V-cycle runs (res > tol, finite, fewer than itmax
// cycles so far).  Records the outcome in MGState; a failure code is sticky.
// With use_handle the decision also drives the graph's while node.
struct MGState {
    int it;                 // V-cycles run in the current solve
    int cont;               // 1: run another V-cycle
    int status;             // first failure: 0, -4 not converged, -5 non-finite
    int last_iters;
    double last_res;
    long long total_iters;  // summed over finished solves
    long long solves;
    unsigned arrive;        // blocks of a fused residual kernel done (reset by the last)
    unsigned arrive_sum;    // blocks of a field-update kernel done (reset by the last)
};

// The decision of the check, by one thread, for the residual max-norm res.
__device__ __forceinline__ void mg_decide(double res, double tol, int itmax, MGState* __restrict__ st,
                                          cudaGraphConditionalHandle handle, int use_handle) {
    int cont = 0;
    if (!(res <= 1.0e308)) {
        if (st->status == 0) st->status = -5;
    } else if (res > tol) {
        if (st->it < itmax) cont = 1;
        else if (st->status == 0) st->status = -4;
    }
    if (st->status == -5 || st->status == -1) cont = 0;  // non-finite data: no further V-cycles
    if (cont) {
        st->it += 1;
    } else {
        st->last_iters = st->it;
        st->last_res = res;
        st->total_iters += st->it;
        st->solves += 1;
        st->it = 0;
    }
    st->cont = cont;
    if (use_handle) cudaGraphSetConditional(handle, cont);
}

static __global__ void __launch_bounds__(1024)
k_mg_check(const double* __restrict__ bmax, int nb, double tol, int itmax, MGState* __restrict__ st,
           cudaGraphConditionalHandle handle, int use_handle) {
    double a = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) a = fmax(a, bmax[i]);
    const double res = block_max(a);
    if (threadIdx.x == 0) mg_decide(res, tol, itmax, st, handle, use_handle);
}

// The check fused into a residual kernel: every block publishes its maximum
// |r| (am, block-uniform) to bmax; the block that arrives last reads all of
// them back from L2 and takes the decision of k_mg_check.
struct CheckArgs {
    double* bmax;
    double tol;
    int itmax;
    MGState* st;
    cudaGraphConditionalHandle handle;
    int use_handle;
    long long* bsum;     // optional: exact block sums of the increments (gauge mode) ...
    long long* sum_out;  // ... added into *sum_out by the last block
};

// Block-wide sum of a 64-bit integer (all threads get the result).
__device__ __forceinline__ long long block_sum_ll(long long v) {
    __shared__ long long shl[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int tid = linear_tid(), lane = tid & 31, wid = tid >> 5;
    __syncthreads();
    if (lane == 0) shl[wid] = v;
    __syncthreads();
    const int nw = (block_threads() + 31) >> 5;
    v = (tid < nw) ? shl[tid] : 0ll;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (tid == 0) shl[0] = v;
    __syncthreads();
    v = shl[0];
    __syncthreads();
    return v;
}

__device__ __forceinline__ void fused_check(float am, const CheckArgs& ck, long long bs = 0) {
    __shared__ int last_s;
    const int tid = linear_tid();
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const int b = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (tid == 0) {
        ck.bmax[b] = (double)am;
        if (ck.sum_out) ck.bsum[b] = bs;
        __threadfence();
        last_s = atomicAdd(&ck.st->arrive, 1u) == (unsigned)(nb - 1);
    }
    __syncthreads();
    if (!last_s) return;
    __threadfence();
    float a = 0.0f;
    long long sacc = 0;
    for (int i = tid; i < nb; i += block_threads()) {
        a = fmaxf(a, (float)__ldcg(ck.bmax + i));
        if (ck.sum_out) sacc += __ldcg(ck.bsum + i);
    }
    a = block_max_f(a);
    if (ck.sum_out) sacc = block_sum_ll(sacc);
    if (tid == 0) {
        ck.st->arrive = 0;
        if (ck.sum_out) *ck.sum_out += sacc;
        mg_decide((double)a, ck.tol, ck.itmax, ck.st, ck.handle, ck.use_handle);
    }
}

// Mixed precision: prediction (Eq. 17), guess z0 and initial residual in one
// launch, with the check fused.  Per point: s = 2 Psi^k - Psi^{k-1} +
// (4pi/h)(q^s - mean), z0 from the history (order ORDER, 0-3), r = s - M z0
// with z0 at the neighbours formed from their history values.  Writes z0,
// the exact residual rfin and its float copy r32.  A non-finite q^s sets
// status to NONFINITE (once per thread, after its points).
template <int ORDER>
__device__ __forceinline__ fix_t z_guess(const fix_t* __restrict__ z1, const fix_t* __restrict__ z2,
                                         const fix_t* __restrict__ z3, int i) {
    if (ORDER == 1) return z1[i];
    if (ORDER == 2) return 2 * z1[i] - z2[i];
    if (ORDER == 3) return 3 * (z1[i] - z2[i]) + z3[i];
    return 0;
}

template <int ORDER>
__global__ void __launch_bounds__(P3_BX * P3_BY, 8)
k_predict_resid_fix(int n, const fix_t* __restrict__ Psik, const fix_t* __restrict__ Psikm1,
                    const float* __restrict__ qs, const double* __restrict__ qsum, double inv_pts, float u,
                    const fix_t* __restrict__ z1, const fix_t* __restrict__ z2, const fix_t* __restrict__ z3,
                    fix_t* __restrict__ z0, fix_t* __restrict__ rfin, float* __restrict__ r32, CheckArgs ck) {
    pdl_wait();
    pdl_trigger();
    __shared__ float mean_s;
    __shared__ fix_t gmean_s;  // mean of the guess (gauge mode), removed from the stored z0
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        mean_s = (float)(qsum[0] * inv_pts);
        const int64_t m = (int64_t)n * n * n;
        // exact sums in fixed point: the guess's sum is the same combination
        // of the history sums (slot m of each buffer); an integer mean is
        // removed and the exact remainder recorded (the V-cycles' increments
        // are added by the residual updates), so the recorded sums never
        // drift from the buffers' true sums
        const fix_t sg = ORDER == 1 ? z1[m] : ORDER == 2 ? 2 * z1[m] - z2[m]
                                                         : ORDER == 3 ? 3 * (z1[m] - z2[m]) + z3[m] : (fix_t)0;
        const fix_t gm = sg / (fix_t)m;
        gmean_s = gm;
        if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) z0[m] = sg - (fix_t)m * gm;
    }
    __syncthreads();
    const fix_t gmean = gmean_s;
    const int x = blockIdx.x * P3_BX + threadIdx.x;
    const int y = blockIdx.y * P3_BY + threadIdx.y;
    float a = 0.0f;
    bool bad = false;
    if (x < n && y < n) {
        const int xm = x == 0 ? n - 1 : x - 1, xp = x == n - 1 ? 0 : x + 1;
        const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
        const float mean = mean_s;
        for (int zz = blockIdx.z; zz < n; zz += gridDim.z) {
            const int zm = zz == 0 ? n - 1 : zz - 1, zp = zz == n - 1 ? 0 : zz + 1;
            const int row = (zz * n + y) * n;
            const int i = row + x;
            const float q = qs[i];
            bad |= !isfinite(q);
            const fix_t s = 2 * Psik[i] - Psikm1[i] + charge_term(q, mean, u);
            const fix_t zc = z_guess<ORDER>(z1, z2, z3, i);
            fix_t nb = 0;
            if (ORDER > 0)
                nb = z_guess<ORDER>(z1, z2, z3, row + xm) + z_guess<ORDER>(z1, z2, z3, row + xp) +
                     z_guess<ORDER>(z1, z2, z3, (zz * n + ym) * n + x) +
                     z_guess<ORDER>(z1, z2, z3, (zz * n + yp) * n + x) +
                     z_guess<ORDER>(z1, z2, z3, (zm * n + y) * n + x) +
                     z_guess<ORDER>(z1, z2, z3, (zp * n + y) * n + x);
            const fix_t res = s - (nb - 6 * zc);  // unchanged by a constant shift of the guess
            z0[i] = zc - gmean;
            rfin[i] = res;
            const float v = fix_to_float(res);
            r32[i] = v;
            a = fmaxf(a, fabsf(v));
        }
    }
    if (bad) atomicCAS(&ck.st->status, 0, -5);
    fused_check(block_max_f(a), ck);
}

// Mixed precision: the V-cycle's float correction e enters once as E =
// fix(e): z += E, and the exact residual is updated without a stencil of z,
//   r_new = s - M (z + E) = r_old - M E,
// with E at the neighbours converted the same way; check fused.  A
// non-finite e sets status to NONFINITE (that point is left unchanged).
static __global__ void __launch_bounds__(P3_BX * P3_BY, 8)  // 32 registers: the 1024 blocks of 128^3 in one wave
k_resid_update_fix(int n, fix_t* __restrict__ z, const float* __restrict__ e, fix_t* __restrict__ rfin,
                   float* __restrict__ r32, CheckArgs ck) {
    pdl_wait();
    pdl_trigger();
    const int x = blockIdx.x * P3_BX + threadIdx.x;
    const int y = blockIdx.y * P3_BY + threadIdx.y;
    float a = 0.0f;
    long long es = 0;  // exact sum of the increments (gauge-mode bookkeeping of z's sum)
    auto fx_of = [](float v) { return fabsf(v) < 8.0e6f ? float_to_fix(v) : (fix_t)0; };
    if (x < n && y < n) {
        const int xm = x == 0 ? n - 1 : x - 1, xp = x == n - 1 ? 0 : x + 1;
        const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
        for (int zz = blockIdx.z; zz < n; zz += gridDim.z) {
            const int zm = zz == 0 ? n - 1 : zz - 1, zp = zz == n - 1 ? 0 : zz + 1;
            const int i = (zz * n + y) * n + x;
            const float ec = e[i];
            if (!(fabsf(ec) < 8.0e6f)) atomicCAS(&ck.st->status, 0, -5);
            const fix_t E = fx_of(ec);
            const int row = (zz * n + y) * n;
            const fix_t nb = fx_of(e[row + xm]) + fx_of(e[row + xp]) + fx_of(e[(zz * n + ym) * n + x]) +
                             fx_of(e[(zz * n + yp) * n + x]) + fx_of(e[(zm * n + y) * n + x]) +
                             fx_of(e[(zp * n + y) * n + x]);
            z[i] += E;
            es += E;
            const fix_t res = rfin[i] - (nb - 6 * E);
            rfin[i] = res;
            const float v = fix_to_float(res);
            r32[i] = v;
            a = fmaxf(a, fabsf(v));
        }
    }
    const float am = block_max_f(a);
    fused_check(am, ck, ck.sum_out ? block_sum_ll(es) : 0ll);
}

// ---------------------------------------------------------------- multigrid
// Red-black Gauss-Seidel half sweep on M e = b: points with (x+y+z)%2 == color
// get e = (sum of neighbours - b)/6.  Thread slot (tx, y, z) handles
// x = 2 tx + parity.  first = 1: the sweep starts from e = 0, so red points
// get -b/6 and black points are cleared (replaces a memset and a sweep).
template <typename T>
__global__ void __launch_bounds__(P3_BX * P3_BY)
k_rbgs(int n, T* __restrict__ e, const T* __restrict__ b, int color, int first) {
    pdl_wait();
    pdl_trigger();
    const int tx = blockIdx.x * P3_BX + threadIdx.x;
    const int y = blockIdx.y * P3_BY + threadIdx.y;
    const int z = blockIdx.z;
    const int x = 2 * tx + ((y + z + color) & 1);
    if (x >= n || y >= n) return;
    const int i = (z * n + y) * n + x;
    if (first) {
        e[i] = -b[i] * (T)(1.0 / 6.0);
        const int xo = x ^ 1;  // the other colour in this pair of x (n even)
        e[i - x + xo] = (T)0;
    } else {
        e[i] = (nb6(e, x, y, z, n) - b[i]) * (T)(1.0 / 6.0);
    }
}

// The first red-black sweep from e = 0 in one launch: red points get -b/6,
// black points (nb6 of the red values - b)/6, with the red values formed
// from b on the fly in the same float operations and order as k_rbgs (each
// product rounded on its own, as the stored values are), so the result
// equals the two half sweeps bit for bit.
template <typename T>
__global__ void __launch_bounds__(P3_BX * P3_BY)
k_rbgs_first(int n, T* __restrict__ e, const T* __restrict__ b) {
    pdl_wait();
    pdl_trigger();
    int x, y, z;
    if (!xyz3(n, x, y, z)) return;
    const int i = (z * n + y) * n + x;
    const T sixth = (T)(1.0 / 6.0);
    if (((x + y + z) & 1) == 0) {
        e[i] = -b[i] * sixth;
        return;
    }
    const int xm = x == 0 ? n - 1 : x - 1, xp = x == n - 1 ? 0 : x + 1;
    const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
    const int zm = z == 0 ? n - 1 : z - 1, zp = z == n - 1 ? 0 : z + 1;
    const int row = (z * n + y) * n;
    auto red = [&](int j) {
        if constexpr (sizeof(T) == 4) return __fmul_rn(-b[j], sixth);
        else return __dmul_rn(-b[j], sixth);
    };
    const T s6 = red(row + xm) + red(row + xp) + red((z * n + ym) * n + x) + red((z * n + yp) * n + x) +
                 red((zm * n + y) * n + x) + red((zp * n + y) * n + x);
    e[i] = (s6 - b[i]) * sixth;
}

// Residual and full-weighting restriction fused: b_c[I] = 4 sum_d w(d)
// (b_f - M e_f)[2I + d], w = prod of (1/4, 1/2, 1/4); the factor 4 is the
// rediscretisation of the dimensionless M on a mesh of twice the spacing.
template <typename T>
__global__ void __launch_bounds__(P3_BX * P3_BY)
k_resid_restrict(int nc, const T* __restrict__ e, const T* __restrict__ b, T* __restrict__ bc) {
    pdl_wait();
    pdl_trigger();
    int X, Y, Z;
    if (!xyz3(nc, X, Y, Z)) return;
    const int n = 2 * nc;
    const T w1[3] = {(T)0.25, (T)0.5, (T)0.25};
    T acc = 0;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
        const int z = wrap_idx(2 * Z + dz, n);
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int y = wrap_idx(2 * Y + dy, n);
            const T wyz = w1[dy + 1] * w1[dz + 1];
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = wrap_idx(2 * X + dx, n);
                const int i = (z * n + y) * n + x;
                acc += wyz * w1[dx + 1] * (b[i] - (nb6(e, x, y, z, n) - (T)6 * e[i]));
            }
        }
    }
    bc[(Z * nc + Y) * nc + X] = (T)4 * acc;
}

// The same residual and full weighting, marched in z: a thread owns the
// coarse column (X, Y) for ZC coarse planes.  It keeps the 3x3 fine points
// around (2X, 2Y) of three consecutive fine planes in registers, with the
// left and right neighbours (x = 2X-2, 2X+2) of the centre plane's rows.
// Per fine plane it loads the next plane's rows as the pairs (2X-2, 2X-1),
// (2X, 2X+1) and the point 2X+2, the rows 2Y-2 and 2Y+2 of the centre plane
// and the 3x3 of b as pairs (n is even, so every pair is aligned), forms the
// nine fine residuals of the plane once (the operand order of nb6) and their
// x-y weighted sum R(z); then
//   bc(X, Y, Z) = 4 (R(2Z-1) / 4 + R(2Z) / 2 + R(2Z+1) / 4).
// The weights are powers of two; only the summation order differs from
// k_resid_restrict.  19 loads per fine plane per thread instead of 27 per
// fine point.
template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

template <typename T, int ZC>
__global__ void __launch_bounds__(P3_BX * P3_BY)
k_resid_restrict_z(int nc, const T* __restrict__ e, const T* __restrict__ b, T* __restrict__ bc) {
    using V2 = typename Vec2<T>::type;
    pdl_wait();
    pdl_trigger();
    const int X = blockIdx.x * P3_BX + threadIdx.x, Y = blockIdx.y * P3_BY + threadIdx.y;
    if (X >= nc || Y >= nc) return;
    const int n = 2 * nc;
    const int Z0 = blockIdx.z * ZC, Z1 = min(Z0 + ZC, nc);
    const int cx = 2 * X, cy = 2 * Y;
    const int xa = cx == 0 ? n - 2 : cx - 2;              // pair (2X-2, 2X-1), wrapped as a pair
    const int xr = cx + 2 >= n ? cx + 2 - n : cx + 2;
    const int ys[3] = {cy == 0 ? n - 1 : cy - 1, cy, cy + 1};
    const int yd = cy < 2 ? cy - 2 + n : cy - 2, yu = cy + 2 >= n ? cy + 2 - n : cy + 2;
    const size_t plane = (size_t)n * n;
    const T w1[3] = {(T)0.25, (T)0.5, (T)0.25};
    T em[3][3], ec[3][3], ep[3][3];  // fine planes z-1, z, z+1: [row][x - 2X + 1]
    T lc[3], rc[3], lp[3], rp[3];    // x = 2X-2 and 2X+2 of the rows of planes z and z+1
    auto load_rows = [&](int z, T (&v)[3][3], T (&l)[3], T (&r)[3]) {
        const T* p = e + (size_t)z * plane;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const V2 a = *reinterpret_cast<const V2*>(p + ys[j] * n + xa);
            const V2 m = *reinterpret_cast<const V2*>(p + ys[j] * n + cx);
            l[j] = a.x;
            v[j][0] = a.y;
            v[j][1] = m.x;
            v[j][2] = m.y;
            r[j] = p[ys[j] * n + xr];
        }
    };
    auto wrapz = [&](int z) { return z < 0 ? z + n : (z >= n ? z - n : z); };
    int f = 2 * Z0 - 1;  // first fine plane
    {
        T l[3], r[3];
        load_rows(wrapz(f - 1), em, l, r);
    }
    load_rows(wrapz(f), ec, lc, rc);
    T r_lo = 0, r_mid = 0;  // R of the fine planes 2Z-1 and 2Z
    for (int k = 0; k <= 2 * (Z1 - Z0); ++k, ++f) {
        const int zf = wrapz(f);
        load_rows(wrapz(f + 1), ep, lp, rp);
        const T* pe = e + (size_t)zf * plane;
        const T* pb = b + (size_t)zf * plane;
        T rd[3], ru[3], bb[3][3];
        {
            const V2 da = *reinterpret_cast<const V2*>(pe + yd * n + xa);
            const V2 dm = *reinterpret_cast<const V2*>(pe + yd * n + cx);
            const V2 ua = *reinterpret_cast<const V2*>(pe + yu * n + xa);
            const V2 um = *reinterpret_cast<const V2*>(pe + yu * n + cx);
            rd[0] = da.y;
            rd[1] = dm.x;
            rd[2] = dm.y;
            ru[0] = ua.y;
            ru[1] = um.x;
            ru[2] = um.y;
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const V2 a = *reinterpret_cast<const V2*>(pb + ys[j] * n + xa);
            const V2 m = *reinterpret_cast<const V2*>(pb + ys[j] * n + cx);
            bb[j][0] = a.y;
            bb[j][1] = m.x;
            bb[j][2] = m.y;
        }
        T R = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const T xm = i == 0 ? lc[j] : ec[j][i - 1];
                const T xp = i == 2 ? rc[j] : ec[j][i + 1];
                const T ym = j == 0 ? rd[i] : ec[j - 1][i];
                const T yp = j == 2 ? ru[i] : ec[j + 1][i];
                const T nb = xm + xp + ym + yp + em[j][i] + ep[j][i];
                R += (w1[j] * w1[i]) * (bb[j][i] - (nb - (T)6 * ec[j][i]));
            }
        }
        if (k & 1) {
            r_mid = R;  // fine plane 2Z
        } else {
            if (k > 0) {  // fine plane 2Z+1 closes coarse plane Z
                const int Z = Z0 + (k >> 1) - 1;
                bc[((size_t)Z * nc + Y) * nc + X] = (T)4 * (w1[0] * r_lo + w1[1] * r_mid + w1[2] * R);
            }
            r_lo = R;  // and opens coarse plane Z + 1
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            lc[j] = lp[j];
            rc[j] = rp[j];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                em[j][i] = ec[j][i];
                ec[j][i] = ep[j][i];
            }
        }
    }
}

// The first red-black sweep from e = 0 (as k_rbgs_first, bit for bit) in
// FP32 with four x points per thread (N % 4 == 0) and ZC z planes per thread,
// every load of the thread's b column (planes z0-1 .. z0+ZC), of the y-1 and
// y+1 rows and of the row-end neighbours issued first; x neighbours of the
// quad from the adjacent lanes.  Red points (x+y+z even) get -b/6, black
// points (the six red neighbours' -b/6 summed in the order x-, x+, y-, y+,
// z-, z+, minus b) / 6.
template <int ZC>
__global__ void __launch_bounds__(P3_BX * P3_BY)
k_rbgs_first4(int n, float* __restrict__ e, const float* __restrict__ b) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x;
    const int qd = blockIdx.x * P3_BX + lane;
    const int x = 4 * qd;
    const int y = blockIdx.y * P3_BY + threadIdx.y;
    const int z0 = blockIdx.z * ZC;
    const bool live = x < n && y < n;
    const int nq = n >> 2;
    const int yy = live ? y : 0, xx = live ? x : 0;
    const int xl = xx == 0 ? n - 1 : xx - 1;
    const int xr = xx + 4 == n ? 0 : xx + 4;
    const int ym = yy == 0 ? n - 1 : yy - 1, yp = yy == n - 1 ? 0 : yy + 1;
    const int plane = n * n;
    const bool lend = lane == 0 || qd - 1 >= nq, rend = lane == P3_BX - 1 || qd + 1 >= nq;
    const float4* b4 = reinterpret_cast<const float4*>(b);
    auto wz = [&](int z) { return z < 0 ? z + n : (z >= n ? z - n : z); };
    float4 col[ZC + 2], am[ZC], bp[ZC];
    float lft[ZC], rgt[ZC];
#pragma unroll
    for (int k = 0; k < ZC + 2; ++k) col[k] = b4[(wz(z0 - 1 + k) * plane + yy * n + xx) >> 2];
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const int z = wz(z0 + k);
        am[k] = b4[(z * plane + ym * n + xx) >> 2];
        bp[k] = b4[(z * plane + yp * n + xx) >> 2];
        lft[k] = lend ? b[z * plane + yy * n + xl] : 0.0f;
        rgt[k] = rend ? b[z * plane + yy * n + xr] : 0.0f;
    }
    const float sixth = (float)(1.0 / 6.0);
    auto red = [&](float v) { return __fmul_rn(-v, sixth); };
#pragma unroll
    for (int k = 0; k < ZC; ++k) {
        const float4 vm = col[k], vc = col[k + 1], vp = col[k + 2], a = am[k], c = bp[k];
        float left = __shfl_up_sync(0xffffffffu, vc.w, 1);
        float right = __shfl_down_sync(0xffffffffu, vc.x, 1);
        if (lend) left = lft[k];
        if (rend) right = rgt[k];
        const int z = z0 + k;
        const bool even0 = ((x + y + z) & 1) == 0;  // parity of the quad's first point
        const float xs[6] = {left, vc.x, vc.y, vc.z, vc.w, right};
        const float ys[4] = {a.x, a.y, a.z, a.w}, yq[4] = {c.x, c.y, c.z, c.w};
        const float zs[4] = {vm.x, vm.y, vm.z, vm.w}, zq[4] = {vp.x, vp.y, vp.z, vp.w};
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool redpt = even0 == ((j & 1) == 0);
            if (redpt) {
                o[j] = red(xs[j + 1]);
            } else {
                const float s6 = red(xs[j]) + red(xs[j + 2]) + red(ys[j]) + red(yq[j]) + red(zs[j]) + red(zq[j]);
                o[j] = (s6 - xs[j + 1]) * sixth;
            }
        }
        if (live && z < n)
            reinterpret_cast<float4*>(e)[(z * plane + yy * n + x) >> 2] = make_float4(o[0], o[1], o[2], o[3]);
    }
}

// One full red-black Gauss-Seidel sweep in one launch (FP32 quads, N % 4 ==
// 0), out of place: colour PA first from the old values in ein, then the
// other colour from the new ones, every point written to eout -- the two
// in-place launches of k_rbgs (PA, then 1 - PA) bit for bit, each point
// formed by the same expression (nb6's operand order, minus b, times 1/6).
// In place it would race: a block reads old second-colour values that its
// neighbours overwrite.  A thread owns a quad of row y and marches ZC planes
// in z; it keeps
// the old rows y-1, y, y+1 of the planes around the current one and the new
// first-colour values of its row at planes z-1, z, z+1 in registers, and
// forms the new first-colour values of rows y-1 and y+1 at plane z itself
// (their old rows y-2 and y+2 loaded), so no value crosses threads but by
// shuffle.  x neighbours come from the adjacent lanes; a warp is one row of
// 32 quads of which lanes 1..30 are written (lanes 0 and 31 are halo, their
// outer points never reach a written value).
template <int PA, int ZC>
__global__ void __launch_bounds__(P3_BX * P3_BY)
k_rbgs_pair4(int n, const float* __restrict__ e, float* __restrict__ eout, const float* __restrict__ b) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x;
    const int nq = n >> 2;
    int qd = (int)blockIdx.x * (P3_BX - 2) + lane - 1;  // quad of this lane (wrapped for loads)
    const bool writer = lane >= 1 && lane <= P3_BX - 2 && qd >= 0 && qd < nq;
    qd = ((qd % nq) + nq) % nq;
    const int x = 4 * qd;
    const int y = (int)blockIdx.y * P3_BY + threadIdx.y;
    const bool live = y < n;
    const int yy = live ? y : 0;
    auto wr = [&](int v) { return v < 0 ? v + n : (v >= n ? v - n : v); };
    const int ym = wr(yy - 1), yp = wr(yy + 1), ymm = wr(yy - 2), ypp = wr(yy + 2);
    const size_t plane = (size_t)n * n;
    auto ld = [&](const float* a, int row, int z) {
        return *reinterpret_cast<const float4*>(a + (size_t)wr(z) * plane + (size_t)row * n + x);
    };
    const float sixth = (float)(1.0 / 6.0);
    // the first colour at the points of quad c (row parity par = (row + z) & 1); the
    // other points keep their old values
    auto first = [&](float4 c, float4 am, float4 ap, float4 zm, float4 zp, float4 bb, int par) {
        const float left = __shfl_up_sync(0xffffffffu, c.w, 1);
        const float right = __shfl_down_sync(0xffffffffu, c.x, 1);
        const float xs[6] = {left, c.x, c.y, c.z, c.w, right};
        const float ya[4] = {am.x, am.y, am.z, am.w}, yb[4] = {ap.x, ap.y, ap.z, ap.w};
        const float za[4] = {zm.x, zm.y, zm.z, zm.w}, zb[4] = {zp.x, zp.y, zp.z, zp.w};
        const float bv[4] = {bb.x, bb.y, bb.z, bb.w};
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (((par + j) & 1) == PA) {
                const float s = xs[j] + xs[j + 2] + ya[j] + yb[j] + za[j] + zb[j];
                o[j] = (s - bv[j]) * sixth;
            } else {
                o[j] = xs[j + 1];
            }
        }
        return make_float4(o[0], o[1], o[2], o[3]);
    };
    const int z0 = blockIdx.z * ZC, z1 = min(z0 + ZC, n);
    // windows: old row y at planes z-1 .. z+2, old rows y-1 and y+1 at z-1 .. z+1,
    // b row y at z, z+1, new first colour of row y at z-1 .. z+1
    float4 r0[4], rm[3], rp[3], bq[2], na[3];
    r0[0] = ld(e, yy, z0 - 2);  // (used only to form na[0])
    r0[1] = ld(e, yy, z0 - 1);
    r0[2] = ld(e, yy, z0);
    r0[3] = ld(e, yy, z0 + 1);
    rm[0] = ld(e, ym, z0 - 1);
    rm[1] = ld(e, ym, z0);
    rp[0] = ld(e, yp, z0 - 1);
    rp[1] = ld(e, yp, z0);
    bq[0] = ld(b, yy, z0 - 1);
    bq[1] = ld(b, yy, z0);
    na[0] = first(r0[1], rm[0], rp[0], r0[0], r0[2], bq[0], (yy + z0 - 1) & 1);
    na[1] = first(r0[2], rm[1], rp[1], r0[1], r0[3], bq[1], (yy + z0) & 1);
    // shift to the loop's indexing: r0 = planes z-1 .. z+1 (+ z+2 loaded in the loop)
    r0[0] = r0[1];
    r0[1] = r0[2];
    r0[2] = r0[3];
    bq[0] = bq[1];
    for (int z = z0; z < z1; ++z) {
        r0[3] = ld(e, yy, z + 2);
        rm[2] = ld(e, ym, z + 1);
        rp[2] = ld(e, yp, z + 1);
        const float4 rmm = ld(e, ymm, z), rpp = ld(e, ypp, z);
        bq[1] = ld(b, yy, z + 1);
        const float4 bm = ld(b, ym, z), bp = ld(b, yp, z);
        na[2] = first(r0[2], rm[2], rp[2], r0[1], r0[3], bq[1], (yy + z + 1) & 1);
        const float4 nam = first(rm[1], rmm, r0[1], rm[0], rm[2], bm, (yy + 1 + z) & 1);
        const float4 nap = first(rp[1], r0[1], rpp, rp[0], rp[2], bp, (yy + 1 + z) & 1);
        // the second colour at row y, plane z from the new first-colour values
        {
            const float4 c = na[1];
            const float left = __shfl_up_sync(0xffffffffu, c.w, 1);
            const float right = __shfl_down_sync(0xffffffffu, c.x, 1);
            const float xs[6] = {left, c.x, c.y, c.z, c.w, right};
            const float ya[4] = {nam.x, nam.y, nam.z, nam.w}, yb[4] = {nap.x, nap.y, nap.z, nap.w};
            const float za[4] = {na[0].x, na[0].y, na[0].z, na[0].w}, zb[4] = {na[2].x, na[2].y, na[2].z, na[2].w};
            const float bv[4] = {bq[0].x, bq[0].y, bq[0].z, bq[0].w};
            const int par = (yy + z) & 1;
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (((par + j) & 1) != PA) {
                    const float s = xs[j] + xs[j + 2] + ya[j] + yb[j] + za[j] + zb[j];
                    o[j] = (s - bv[j]) * sixth;
                } else {
                    o[j] = xs[j + 1];
                }
            }
            if (writer && live)
                *reinterpret_cast<float4*>(eout + (size_t)z * plane + (size_t)yy * n + x) =
                    make_float4(o[0], o[1], o[2], o[3]);
        }
        r0[0] = r0[1];
        r0[1] = r0[2];
        r0[2] = r0[3];
        rm[0] = rm[1];
        rm[1] = rm[2];
        rp[0] = rp[1];
        rp[1] = rp[2];
        bq[0] = bq[1];
        na[0] = na[1];
        na[1] = na[2];
    }
}

// Trilinear prolongation and correction e_f += P e_c in FP32 with four x
// points and the two z planes 2Z, 2Z+1 per thread (N % 4 == 0): the 12
// coarse values of a quad pair are loaded once and every output is formed
// by prolong_at's expression.
static __global__ void __launch_bounds__(P3_BX * P3_BY)
k_prolong_add4(int n, const float* __restrict__ ec, float* __restrict__ ef) {
    pdl_wait();
    pdl_trigger();
    const int qd = blockIdx.x * P3_BX + threadIdx.x;
    const int x = 4 * qd;
    const int y = blockIdx.y * P3_BY + threadIdx.y;
    const int Z = blockIdx.z;
    const int nc = n >> 1;
    if (x >= n || y >= n) return;
    const int cxa = x >> 1, cxb = cxa + 1, cxc = cxa + 2 >= nc ? cxa + 2 - nc : cxa + 2;  // 2q, 2q+1, 2q+2
    const int y0 = y >> 1, y1 = (y & 1) ? (y0 + 1 == nc ? 0 : y0 + 1) : y0;
    const float ay = (y & 1) ? 0.5f : 1.0f, by = (y & 1) ? 0.5f : 0.0f;
    const int Zp = Z + 1 == nc ? 0 : Z + 1;
    float c[2][2][3];  // [z: Z, Z+1][y: y0, y1][x: 2q, 2q+1, 2q+2]
    const int zz[2] = {Z, Zp}, yyv[2] = {y0, y1};
#pragma unroll
    for (int iz = 0; iz < 2; ++iz)
#pragma unroll
        for (int iy = 0; iy < 2; ++iy) {
            const float* row = ec + (zz[iz] * nc + yyv[iy]) * nc;
            c[iz][iy][0] = row[cxa];
            c[iz][iy][1] = row[cxb];
            c[iz][iy][2] = row[cxc];
        }
    const int plane = n * n;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int z = 2 * Z + k;
        const float az = k ? 0.5f : 1.0f, bz = k ? 0.5f : 0.0f;
        const int z1 = k ? 1 : 0;  // second z plane index into c (Z+1 for odd z, Z again for even)
        float4* dst = reinterpret_cast<float4*>(ef + z * plane + y * n + x);
        float4 v = *dst;
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i0 = j >> 1, i1 = (j & 1) ? i0 + 1 : i0;
            const float ax = (j & 1) ? 0.5f : 1.0f, bx = (j & 1) ? 0.5f : 0.0f;
            o[j] = az * (ay * (ax * c[0][0][i0] + bx * c[0][0][i1]) + by * (ax * c[0][1][i0] + bx * c[0][1][i1])) +
                   bz * (ay * (ax * c[z1][0][i0] + bx * c[z1][0][i1]) + by * (ax * c[z1][1][i0] + bx * c[z1][1][i1]));
        }
        v.x += o[0];
        v.y += o[1];
        v.z += o[2];
        v.w += o[3];
        *dst = v;
    }
}

// Trilinear prolongation and correction on the fine level: e_f += P e_c.
template <typename T>
__device__ __forceinline__ T prolong_at(const T* __restrict__ ec, int nc, int x, int y, int z) {
    const int x0 = x >> 1, y0 = y >> 1, z0 = z >> 1;
    const int x1 = (x & 1) ? (x0 + 1 == nc ? 0 : x0 + 1) : x0;
    const int y1 = (y & 1) ? (y0 + 1 == nc ? 0 : y0 + 1) : y0;
    const int z1 = (z & 1) ? (z0 + 1 == nc ? 0 : z0 + 1) : z0;
    const T ax = (x & 1) ? (T)0.5 : (T)1, bx = (x & 1) ? (T)0.5 : (T)0;
    const T ay = (y & 1) ? (T)0.5 : (T)1, by = (y & 1) ? (T)0.5 : (T)0;
    const T az = (z & 1) ? (T)0.5 : (T)1, bz = (z & 1) ? (T)0.5 : (T)0;
    const T* p00 = ec + (z0 * nc + y0) * nc;
    const T* p01 = ec + (z0 * nc + y1) * nc;
    const T* p10 = ec + (z1 * nc + y0) * nc;
    const T* p11 = ec + (z1 * nc + y1) * nc;
    return az * (ay * (ax * p00[x0] + bx * p00[x1]) + by * (ax * p01[x0] + bx * p01[x1])) +
           bz * (ay * (ax * p10[x0] + bx * p10[x1]) + by * (ax * p11[x0] + bx * p11[x1]));
}

template <typename T>
__global__ void __launch_bounds__(P3_BX * P3_BY)
k_prolong_add(int n, const T* __restrict__ ec, T* __restrict__ ef) {
    pdl_wait();
    pdl_trigger();
    int x, y, z;
    if (!xyz3(n, x, y, z)) return;
    ef[(z * n + y) * n + x] += prolong_at(ec, n >> 1, x, y, z);
}

// ---------------------------------------------------------------- coarse solve
// Exact solve of M e = b on the coarsest level (n <= 64) by separable real
// Hartley transforms.  H[k][x] = cos(2 pi k x / n) + sin(2 pi k x / n) is
// symmetric with H H = n I, and H C H = n diag(lambda) for every symmetric
// periodic 1D stencil C; the 7-point M is a sum of one such stencil per
// axis, so M = H3 diag(Lambda) H3 / n^3 with H3 = Hz (x) Hy (x) Hx and
// Lambda(k) = -4 sum_axes sin^2(pi k_axis / n).  The pseudo-inverse solve is
//   e = H3 (D o (H3 b)),  D = 1 / (Lambda n^3), and 0 at k = 0,
// the zero-mean solution (the mean of b is dropped).  Three launches of n
// blocks: the x and y transforms of each z plane (k_coarse_xy), the z
// transform, scaling and inverse z transform of each plane of constant ky
// (k_coarse_z), and the inverse x and y transforms (k_coarse_xy again: the
// transforms of different axes commute).  Arrays are staged in shared memory
// padded to nP = 4 ceil(n/4) with zeros; each thread forms a 4 x 4 tile of
// outputs (16 FMAs per 8 shared-memory loads).
constexpr int kCoarseMax = 64;
constexpr int kCoarseThreads = 256;

template <typename T>
__device__ __forceinline__ void ld4s(const T* p, T v[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 f = *reinterpret_cast<const float4*>(p);
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
    } else {
        v[0] = p[0]; v[1] = p[1]; v[2] = p[2]; v[3] = p[3];
    }
}

template <typename T>
__device__ __forceinline__ void st4s(T* p, T a, T b, T c, T d) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
    } else {
        p[0] = a; p[1] = b; p[2] = c; p[3] = d;
    }
}

// Stage the n x n table H and the n x n slice src (row stride sstride) into
// shared memory, zero-padded to nP x nP.
// Every load is issued before the first store (one memory round trip).
template <typename T>
__device__ __forceinline__ void coarse_stage(int n, int nP, const T* __restrict__ H, const T* __restrict__ src,
                                             int64_t sstride, T* sH, T* sA) {
    constexpr int kPer = (kCoarseMax * kCoarseMax + kCoarseThreads - 1) / kCoarseThreads;
    T h[kPer], a[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int i = threadIdx.x + k * kCoarseThreads;
        const int r = i / nP, c = i - r * nP;
        h[k] = (i < nP * nP && r < n && c < n) ? H[r * n + c] : (T)0;
    }
    pdl_wait();  // H is constant; src is the predecessor's output
    pdl_trigger();
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int i = threadIdx.x + k * kCoarseThreads;
        const int r = i / nP, c = i - r * nP;
        a[k] = (i < nP * nP && r < n && c < n) ? src[r * sstride + c] : (T)0;
    }
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int i = threadIdx.x + k * kCoarseThreads;
        if (i < nP * nP) {
            sH[i] = h[k];
            sA[i] = a[k];
        }
    }
}

// out[r][c] = sum_m L[m][r] R[m][c] over m < nP (L, R in shared memory with
// row length nP; L symmetric use: L[m][r] = H[r][m]); tile (r0, c0) of 4 x 4.
template <typename T>
__device__ __forceinline__ void coarse_tile(int nP, const T* L, const T* R, int r0, int c0, T acc[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
#pragma unroll 4
    for (int m = 0; m < nP; ++m) {
        T l[4], r[4];
        ld4s(L + m * nP + r0, l);
        ld4s(R + m * nP + c0, r);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += l[i] * r[j];
    }
}

// y then x transform of plane z = blockIdx.x: out[z] = Hy A Hx (A = in[z]).
// The y pass stores its result transposed (float4 per thread along its
// rows, lanes along rows: conflict-free), so both passes read rows.
template <typename T>
__global__ void __launch_bounds__(kCoarseThreads)
k_coarse_xy(int n, const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ H) {
    extern __shared__ __align__(16) unsigned char coarse_smem[];
    const int nP = (n + 3) & ~3, t4 = nP >> 2;
    T* sH = reinterpret_cast<T*>(coarse_smem);
    T* sA = sH + nP * nP;
    T* sB = sA + nP * nP;
    const int64_t plane = (int64_t)n * n;
    const int z = blockIdx.x;
    coarse_stage(n, nP, H, in + z * plane, n, sH, sA);
    __syncthreads();
    const int tile = threadIdx.x;
    const bool act = tile < t4 * t4;
    T acc[4][4];
    // y pass: C[j][x] = sum_y H[y][j] A[y][x]; sB[x][j] = C[j][x]
    if (act) {
        const int tj = tile % t4, tx = tile / t4;
        coarse_tile(nP, sH, sA, 4 * tj, 4 * tx, acc);
#pragma unroll
        for (int c = 0; c < 4; ++c) st4s(sB + (4 * tx + c) * nP + 4 * tj, acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
    }
    __syncthreads();
    // x pass: out[j][k] = sum_x C[j][x] H[x][k] = sum_x sB[x][j] sH[x][k]
    if (act) {
        const int tj = tile / t4, tk = tile % t4;
        coarse_tile(nP, sB, sH, 4 * tj, 4 * tk, acc);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = 4 * tj + i;
            if (r >= n) break;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int k = 4 * tk + c;
                if (k < n) out[z * plane + (int64_t)r * n + k] = acc[i][c];
            }
        }
    }
}

// For ky = blockIdx.x: forward z transform, scaling by D, inverse z transform
// of the slice t[z][ky][kx] (in place).
template <typename T>
__global__ void __launch_bounds__(kCoarseThreads)
k_coarse_z(int n, T* __restrict__ t, const T* __restrict__ H, const T* __restrict__ D) {
    extern __shared__ __align__(16) unsigned char coarse_smem[];
    const int nP = (n + 3) & ~3, t4 = nP >> 2;
    T* sH = reinterpret_cast<T*>(coarse_smem);
    T* sA = sH + nP * nP;
    T* sB = sA + nP * nP;
    const int64_t plane = (int64_t)n * n;
    const int j = blockIdx.x;
    const int tile = threadIdx.x, tz = tile / t4, tk = tile - tz * t4;
    const bool act = tile < t4 * t4;
    // this thread's 16 scale factors, loaded with the staging
    T dsc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int kz = 4 * tz + i, kx = 4 * tk + c;
            dsc[i][c] = (act && kz < n && kx < n) ? D[((int64_t)kz * n + j) * n + kx] : (T)0;
        }
    coarse_stage(n, nP, H, t + (int64_t)j * n, plane, sH, sA);  // sA[z][kx]
    __syncthreads();
    T acc[4][4];
    // U[kz][kx] = sum_z H[z][kz] A[z][kx], scaled by D[kz][ky][kx]
    if (act) {
        coarse_tile(nP, sH, sA, 4 * tz, 4 * tk, acc);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int kz = 4 * tz + i;
            st4s(sB + kz * nP + 4 * tk, acc[i][0] * dsc[i][0], acc[i][1] * dsc[i][1], acc[i][2] * dsc[i][2],
                 acc[i][3] * dsc[i][3]);
        }
    }
    __syncthreads();
    // V[z][kx] = sum_kz H[kz][z] U[kz][kx]
    if (act) {
        coarse_tile(nP, sH, sB, 4 * tz, 4 * tk, acc);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int z = 4 * tz + i;
            if (z >= n) break;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int kx = 4 * tk + c;
                if (kx < n) t[z * plane + (int64_t)j * n + kx] = acc[i][c];
            }
        }
    }
}

// Shared memory of the coarse kernels for a level of n points per axis.
inline size_t coarse_smem_bytes(int n, size_t tb) {
    const size_t nP = (size_t)((n + 3) & ~3);
    return 3 * nP * nP * tb;
}

// ---------------------------------------------------------------- spectral smoothing by FFT
// (I + cM)^K q for meshes of n = 32, 64 or 128 points per axis (powers of two
// whose n x n plane fits in shared memory).  The operator is the separable
// Hartley diagonalisation of the coarse solve, q^s = H3 (S o (H3 q)) with
// S(k) = (1 + c lambda_k)^K / n^3, but each 1D Hartley transform takes
// O(n log n) operations: two real lines a, b packed as z = a + ib go through
// one complex FFT Z, and with A = (Z[k] + conj Z[n-k]) / 2 (the DFT of a),
// B = (Z[k] - conj Z[n-k]) / 2i (that of b), the Hartley coefficients
// Re A - Im A and Re B - Im B are
//   Ha[k] = (Re Z[k] - Im Z[k] + Re Z[n-k] + Im Z[n-k]) / 2,
//   Hb[k] = (Re Z[k] + Im Z[k] - Re Z[n-k] + Im Z[n-k]) / 2.
// One warp transforms one pair of lines: lane l holds points l + 32 j
// (j < n / 32) in registers; the radix-2 decimation-in-frequency stages of
// half-size 32 and more run inside the lane, those of half-size 16 .. 1
// across lanes by shuffles.  The forward transforms (decimation in
// frequency) leave the coefficients in bit-reversed order, the inverse ones
// (decimation in time) take them so and return natural order: the scaling
// table is stored bit-reversed in all three indices, and nothing is ever
// reordered.  The split's partner Z[n - k] is in another lane and comes by
// one shuffle per register.  The kernels form 2 Ha and 2 Hb (the halving
// is left to the scaling table, which carries 1/64 for the six transforms).
// Twiddles exp(-2 pi i k / n), k < n / 2, are FP64 values rounded once to
// FP32; each lane keeps the ones it uses in registers.  Three launches of n
// blocks: forward x and y transforms of each z plane (k_fht_xy), forward z
// transform, scaling and inverse z transform of each plane of constant ky
// (k_fht_z), and the inverse x and y transforms (k_fht_xy), which also
// write the compensated sum of each output plane.
//
// Shared-memory layout of an n x n plane: element (r, c) at
// r n + (c ^ (r mod 32)) (k_fht_xy's row pass reads its rows straight from
// global memory and writes them so).  Rows stay 16-byte
// aligned (the XOR keeps each group of four within its 16 bytes), and a warp
// reading or writing 32 consecutive elements of a row or of a column touches
// 32 distinct banks.
constexpr int kFhtMaxN = 128;

template <int R>
__host__ __device__ constexpr int fht_threads() { return R == 1 ? 512 : 1024; }

template <int R>
__device__ __forceinline__ int fht_at(int r, int c) { return r * (32 * R) + (c ^ (r & 31)); }

// element p of line `line`: a row (COL false) or a column (COL true)
template <int R, bool COL>
__device__ __forceinline__ int fht_line(int line, int p) { return COL ? fht_at<R>(p, line) : fht_at<R>(line, p); }

// g[e] = f[e ^ x]: the order of a row's four elements inside their 16 bytes
__device__ __forceinline__ float4 fht_perm4(float4 f, int x) {
    if (x & 1) f = make_float4(f.y, f.x, f.w, f.z);
    if (x & 2) f = make_float4(f.z, f.w, f.x, f.y);
    return f;
}

__device__ __forceinline__ float2 fht_cmul(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}

// Line length n = 32 R with R = Q R2: Q = 3 or 5 for a mixed-radix length
// (192, 320, 384), else 1; R2 a power of two.  The radix-2 part transforms
// m = 32 R2 points.
template <int R>
struct FhtShape {
    static constexpr int Q = R % 3 == 0 ? 3 : R % 5 == 0 ? 5 : 1;
    static constexpr int R2 = R / Q;
};

// The twiddles of one lane.  Radix-2 part (m points): stage of half-size
// 32 M (M = R2/2 .. 1), register pair (j, j + M), j mod 2M = j' < M:
// in[M - 1 + j'] = W_{64M}^(lane + 32 j'); cross-lane stage of half-size
// h = 16 >> s (s < 4): x[s] = W_{2h}^(lane mod h) on the lane with bit h set,
// 1 on its partner (half-size 1 needs none).  Radix-Q step: rq[j1 (Q-1) +
// k - 1] = W_n^((lane + 32 j1) k), om[j] = exp(-2 pi i j / Q).  The table tw
// holds W_n^t, t < n/2, then (Q > 1) the Q roots of unity.
template <int R>
struct FhtTw {
    static constexpr int Q = FhtShape<R>::Q, R2 = FhtShape<R>::R2;
    float2 in[R2 > 1 ? R2 - 1 : 1];
    float2 x[4];
    float2 rq[Q > 1 ? R2 * (Q - 1) : 1];
    float2 om[Q > 1 ? Q : 1];
};

template <int R>
__device__ __forceinline__ void fht_twiddles(FhtTw<R>& t, const float2* __restrict__ tw, int lane) {
    constexpr int n = 32 * R, Q = FhtShape<R>::Q, R2 = FhtShape<R>::R2, m = 32 * R2;
    // W_m^k = W_n^(Q k)
#pragma unroll
    for (int M = R2 / 2; M >= 1; M >>= 1)
#pragma unroll
        for (int j = 0; j < M; ++j) t.in[M - 1 + j] = tw[Q * (lane + 32 * j) * (m / (64 * M))];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int h = 16 >> s;
        t.x[s] = (lane & h) ? tw[Q * (lane & (h - 1)) * (m / (2 * h))] : make_float2(1.f, 0.f);
    }
    if constexpr (Q > 1) {
#pragma unroll
        for (int j1 = 0; j1 < R2; ++j1)
#pragma unroll
            for (int k = 1; k < Q; ++k) {
                const int e = (lane + 32 * j1) * k;  // < n; W_n^(e) = -W_n^(e - n/2) past n/2
                const float2 w = tw[e < n / 2 ? e : e - n / 2];
                t.rq[j1 * (Q - 1) + k - 1] = e < n / 2 ? w : make_float2(-w.x, -w.y);
            }
#pragma unroll
        for (int j = 0; j < Q; ++j) t.om[j] = tw[n / 2 + j];
    }
}

// In-place radix-2 DIF FFT of m = 32 R2 points held as v[j] = z[lane + 32 j];
// on return v[j] holds Z[rev(lane + 32 j)] (log2 m-bit reversal).
template <int R2>
__device__ __forceinline__ void warp_fft_dif_p2(float2 (&v)[R2], const float2* tin, const float2* tx, int lane) {
#pragma unroll
    for (int M = R2 / 2; M >= 1; M >>= 1)
#pragma unroll
        for (int j = 0; j < R2; ++j)
            if ((j & M) == 0) {
                const float2 a = v[j], b = v[j + M];
                v[j] = make_float2(a.x + b.x, a.y + b.y);
                v[j + M] = fht_cmul(make_float2(a.x - b.x, a.y - b.y), tin[M - 1 + (j & (2 * M - 1))]);
            }
    // lane pairs (l, l ^ h): the lane with bit h set holds z[i + h] and forms
    // (z[i] - z[i + h]) W_{2h}^(i mod 2h), its partner z[i] + z[i + h]
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int h = 16 >> s;
        const float sg = (lane & h) ? -1.f : 1.f;
#pragma unroll
        for (int j = 0; j < R2; ++j) {
            const float ox = __shfl_xor_sync(0xffffffffu, v[j].x, h);
            const float oy = __shfl_xor_sync(0xffffffffu, v[j].y, h);
            const float2 d = make_float2(fmaf(sg, v[j].x, ox), fmaf(sg, v[j].y, oy));
            v[j] = s < 4 ? fht_cmul(d, tx[s]) : d;
        }
    }
}

// In-place radix-2 DIT FFT: v[j] holds X[rev(lane + 32 j)] on entry and
// Y[lane + 32 j] = sum_k X[k] W_m^(k (lane + 32 j)) on return.  The stages
// of the DIF transform in reverse order, each twiddle applied to the upper
// input before its butterfly.
template <int R2>
__device__ __forceinline__ void warp_fft_dit_p2(float2 (&v)[R2], const float2* tin, const float2* tx, int lane) {
#pragma unroll
    for (int s = 4; s >= 0; --s) {
        const int h = 16 >> s;
        const float sg = (lane & h) ? -1.f : 1.f;
#pragma unroll
        for (int j = 0; j < R2; ++j) {
            const float2 u = s < 4 ? fht_cmul(v[j], tx[s]) : v[j];
            const float ox = __shfl_xor_sync(0xffffffffu, u.x, h);
            const float oy = __shfl_xor_sync(0xffffffffu, u.y, h);
            v[j] = make_float2(fmaf(sg, u.x, ox), fmaf(sg, u.y, oy));
        }
    }
#pragma unroll
    for (int M = 1; M <= R2 / 2; M <<= 1)
#pragma unroll
        for (int j = 0; j < R2; ++j)
            if ((j & M) == 0) {
                const float2 a = v[j], b = fht_cmul(v[j + M], tin[M - 1 + (j & (2 * M - 1))]);
                v[j] = make_float2(a.x + b.x, a.y + b.y);
                v[j + M] = make_float2(a.x - b.x, a.y - b.y);
            }
}

__device__ __forceinline__ float2 fht_cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// DIF FFT of n = 32 R points held as v[j] = z[lane + 32 j].  Q = 1: radix 2,
// position p holds Z[rev(p)].  Q > 1: first the radix-Q step across the
// registers j1 + R2 j2 (points q + m j2, q = lane + 32 j1): Y_k[q] =
// W_n^(q k) sum_j2 z[q + m j2] W_Q^(j2 k) into register j1 + R2 k, then the
// m-point radix-2 transform of each Y_k; position q' + m k (q' = lane +
// 32 j1) holds Z[k + Q rev_m(q')].
template <int R>
__device__ __forceinline__ void warp_fft_dif(float2 (&v)[R], const FhtTw<R>& t, int lane) {
    constexpr int Q = FhtShape<R>::Q, R2 = FhtShape<R>::R2;
    if constexpr (Q == 1) {
        warp_fft_dif_p2<R>(v, t.in, t.x, lane);
    } else {
#pragma unroll
        for (int j1 = 0; j1 < R2; ++j1) {
            float2 xs[Q];
#pragma unroll
            for (int j2 = 0; j2 < Q; ++j2) xs[j2] = v[j1 + R2 * j2];
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                float2 y = xs[0];
#pragma unroll
                for (int j2 = 1; j2 < Q; ++j2) y = fht_cadd(y, fht_cmul(xs[j2], t.om[(j2 * k) % Q]));
                v[j1 + R2 * k] = k ? fht_cmul(y, t.rq[j1 * (Q - 1) + k - 1]) : y;
            }
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            float2 g[R2];
#pragma unroll
            for (int j1 = 0; j1 < R2; ++j1) g[j1] = v[j1 + R2 * k];
            warp_fft_dif_p2<R2>(g, t.in, t.x, lane);
#pragma unroll
            for (int j1 = 0; j1 < R2; ++j1) v[j1 + R2 * k] = g[j1];
        }
    }
}

// DIT FFT: v holds X in warp_fft_dif's output order on entry and
// Y[lane + 32 j] = sum_f X[f] W_n^(f (lane + 32 j)) on return.  Q > 1: the
// m-point radix-2 transform of each group k, then per q the twiddle
// W_n^(q k) and the radix-Q step across the groups.
template <int R>
__device__ __forceinline__ void warp_fft_dit(float2 (&v)[R], const FhtTw<R>& t, int lane) {
    constexpr int Q = FhtShape<R>::Q, R2 = FhtShape<R>::R2;
    if constexpr (Q == 1) {
        warp_fft_dit_p2<R>(v, t.in, t.x, lane);
    } else {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            float2 g[R2];
#pragma unroll
            for (int j1 = 0; j1 < R2; ++j1) g[j1] = v[j1 + R2 * k];
            warp_fft_dit_p2<R2>(g, t.in, t.x, lane);
#pragma unroll
            for (int j1 = 0; j1 < R2; ++j1) v[j1 + R2 * k] = g[j1];
        }
#pragma unroll
        for (int j1 = 0; j1 < R2; ++j1) {
            float2 gs[Q];
#pragma unroll
            for (int k = 0; k < Q; ++k)
                gs[k] = k ? fht_cmul(v[j1 + R2 * k], t.rq[j1 * (Q - 1) + k - 1]) : v[j1 + R2 * k];
#pragma unroll
            for (int j2 = 0; j2 < Q; ++j2) {
                float2 y = gs[0];
#pragma unroll
                for (int k = 1; k < Q; ++k) y = fht_cadd(y, fht_cmul(gs[k], t.om[(k * j2) % Q]));
                v[j1 + R2 * j2] = y;
            }
        }
    }
}

// Shared-memory word at byte offset off of the kernel's dynamic shared memory.
__device__ __forceinline__ float& fht_s(unsigned off) {
    extern __shared__ __align__(16) unsigned char fht_smem[];
    return *reinterpret_cast<float*>(fht_smem + off);
}

// Highest set bit of x > 0 (as a value); 0 for x = 0.
__host__ __device__ constexpr int fht_hibit(int x) {
    int h = x ? 1 : 0;
    while (h && h <= x / 2) h <<= 1;
    return h;
}

// Hartley transforms, times 2, of two lines held as v[j] = (a, b) at point
// lane + 32 j; on return v[j] = (2 Ha, 2 Hb) at position lane + 32 j.
// Forward (INV false): points in natural order, coefficients in
// warp_fft_dif's order.  Inverse: points in that order, coefficients in
// natural order (DIT).  The split pairs each Z[f] with Z[n - f], which
// another lane holds:
//  - DIF output, position p = l + 32 j1 + m k (register j = j1 + R2 k, Z[f]
//    with f = k + Q rev_m(l + 32 j1)): for k = 0 the partner is the radix-2
//    one, p ^ (hibit(p) - 1), i.e. lane l ^ (hibit(l) - 1) for j1 = 0, else
//    lane l ^ 31 and register j1 ^ (hibit(j1) - 1); for k > 0 it is
//    f' = (Q - k) + Q (m - 1 - rev_m(l + 32 j1)): lane l ^ 31, register
//    (j1 ^ (R2 - 1)) + R2 (Q - k);
//  - DIT output, position m = l + 32 j: n - m is lane 32 - l, register
//    R - 1 - j for l > 0, and register (R - j) mod R of lane 0 itself.
// All 32 lanes of a warp call it.
template <int R, bool INV>
__device__ __forceinline__ void fht_pair(float2 (&v)[R], const FhtTw<R>& t, int lane) {
    float2 w[R];
    if constexpr (INV) {
        warp_fft_dit<R>(v, t, lane);
        const int src = (32 - lane) & 31;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            w[j].x = __shfl_sync(0xffffffffu, v[R - 1 - j].x, src);
            w[j].y = __shfl_sync(0xffffffffu, v[R - 1 - j].y, src);
            if (lane == 0) w[j] = v[(R - j) % R];
        }
    } else {
        warp_fft_dif<R>(v, t, lane);
        constexpr int Q = FhtShape<R>::Q, R2 = FhtShape<R>::R2;
        const int src0 = lane ? lane ^ ((1 << (31 - __clz(lane))) - 1) : 0;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const int j1 = j % R2, k = j / R2;
            const int jp = k ? (j1 ^ (R2 - 1)) + R2 * (Q - k) : j1 ? j1 ^ (fht_hibit(j1) - 1) : 0;
            const int src = (k || j1) ? lane ^ 31 : src0;
            w[j].x = __shfl_sync(0xffffffffu, v[jp].x, src);
            w[j].y = __shfl_sync(0xffffffffu, v[jp].y, src);
        }
    }
#pragma unroll
    for (int j = 0; j < R; ++j)
        v[j] = make_float2((v[j].x - v[j].y) + (w[j].x + w[j].y), (v[j].x + v[j].y) + (w[j].y - w[j].x));
}

// The same for two lines in shared memory: point lane + 32 j of line a read
// at byte ia + j JS, its coefficient written at oa + j JS (likewise for b).
template <int R, bool INV, unsigned JS>
__device__ __forceinline__ void warp_fht2(unsigned ia, unsigned ib, unsigned oa, unsigned ob, const FhtTw<R>& t,
                                          int lane) {
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = make_float2(fht_s(ia + j * JS), fht_s(ib + j * JS));
    fht_pair<R, INV>(v, t, lane);
    __syncwarp();  // every lane has read its points before any writes in place
#pragma unroll
    for (int j = 0; j < R; ++j) {
        fht_s(oa + j * JS) = v[j].x;
        fht_s(ob + j * JS) = v[j].y;
    }
}

// Row pass: each warp's row pairs of the plane at src read straight from
// global memory (all of them before the first transform), transformed, and
// written swizzled into the plane at shared byte 0.
template <int R, bool INV>
__device__ __forceinline__ void fht_rows(const float* __restrict__ src, const FhtTw<R>& t, int warp, int lane) {
    constexpr int n = 32 * R, W = fht_threads<R>() / 32, NT = n / 2 / W;
    static_assert(NT * W == n / 2, "row pairs per warp");
    float2 v[NT][R];
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        const int r = 2 * (warp + i * W);
#pragma unroll
        for (int j = 0; j < R; ++j)
            v[i][j] = make_float2(src[r * n + lane + 32 * j], src[(r + 1) * n + lane + 32 * j]);
    }
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        const int r = 2 * (warp + i * W);
        fht_pair<R, INV>(v[i], t, lane);
        const unsigned oa = 4u * (unsigned)(r * n + (lane ^ (r & 31)));
        const unsigned ob = 4u * (unsigned)((r + 1) * n + (lane ^ ((r + 1) & 31)));
#pragma unroll
        for (int j = 0; j < R; ++j) {
            fht_s(oa + 128u * j) = v[i][j].x;
            fht_s(ob + 128u * j) = v[i][j].y;
        }
    }
}

// Column pass over the swizzled plane at byte 0, in place.
template <int R, bool INV>
__device__ __forceinline__ void fht_cols(const FhtTw<R>& t, int warp, int lane) {
    constexpr int n = 32 * R, W = fht_threads<R>() / 32;
    for (int p = warp; p < n / 2; p += W) {
        const int c = 2 * p;
        const unsigned a = 4u * (unsigned)(lane * n + (c ^ lane)), b = 4u * (unsigned)(lane * n + ((c + 1) ^ lane));
        warp_fht2<R, INV, 128u * n>(a, b, a, b, t, lane);
    }
}

// Shared memory of the FFT smoothing kernels at n points per axis: the
// plane, and for k_fht_z the slice of S.
inline size_t fht_smem_bytes(int n) { return (size_t)n * n * sizeof(float); }
inline size_t fht_z_smem_bytes(int n) { return 2 * fht_smem_bytes(n); }

// x and y transforms of z plane blockIdx.x: out[z] = 4 Hy in[z] Hx, forward
// (natural order in, bit-reversed in x and y out) or inverse (the reverse).
// With partial != nullptr, partial[blockIdx.x] gets the compensated sum of
// the output plane and the last block to finish writes their sum (fixed
// order) to *sum_out.
template <int R, bool INV>
__global__ void __launch_bounds__(fht_threads<R>())
k_fht_xy(const float* __restrict__ in, float* __restrict__ out, const float2* __restrict__ tw,
         double* __restrict__ partial, unsigned* __restrict__ arrive, double* __restrict__ sum_out) {
    constexpr int n = 32 * R, T = fht_threads<R>(), Q = n * n / 4, PER = (Q + T - 1) / T;
    extern __shared__ __align__(16) unsigned char fht_smem[];
    float* s = reinterpret_cast<float*>(fht_smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    FhtTw<R> t;
    fht_twiddles<R>(t, tw, lane);  // constant: before the wait
    const int64_t base = (int64_t)blockIdx.x * Q;
    pdl_wait();
    pdl_trigger();
    fht_rows<R, INV>(in + base * 4, t, warp, lane);
    __syncthreads();
    fht_cols<R, INV>(t, warp, lane);
    __syncthreads();
    float4* dst = reinterpret_cast<float4*>(out) + base;
    float acc_s = 0.f, acc_c = 0.f;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * T, r = 4 * i / n, c = 4 * i % n;
        if (i < Q) {
            const float4 v = fht_perm4(*reinterpret_cast<const float4*>(s + r * n + (c ^ (r & 28))), r & 3);
            dst[i] = v;
            if (partial) {
                two_sum_add(acc_s, acc_c, v.x);
                two_sum_add(acc_s, acc_c, v.y);
                two_sum_add(acc_s, acc_c, v.z);
                two_sum_add(acc_s, acc_c, v.w);
            }
        }
    }
    if (partial) sum_last_block((double)acc_s + (double)acc_c, partial, arrive, sum_out);
}

// For ky = blockIdx.x: forward z transform of the slice t[z][ky][x] (rows
// z, columns x of a swizzled plane in shared memory), scaling by S (laid
// out like t, bit-reversed in all three indices; its slice copied
// asynchronously into a second shared plane while the transform runs, each
// 16-byte group at its swizzled position, in natural order), and the
// inverse z transform, in place.
template <int R>
__global__ void __launch_bounds__(fht_threads<R>())
k_fht_z(float* __restrict__ tz, const float2* __restrict__ tw, const float* __restrict__ S) {
    constexpr int n = 32 * R, T = fht_threads<R>(), Q = n * n / 4, PER = (Q + T - 1) / T;
    extern __shared__ __align__(16) unsigned char fht_smem[];
    float* s = reinterpret_cast<float*>(fht_smem);
    float* ss = s + n * n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t ky = blockIdx.x;
    FhtTw<R> t;
    fht_twiddles<R>(t, tw, lane);
#pragma unroll
    for (int k = 0; k < PER; ++k) {  // S is constant: before the wait
        const int i = tid + k * T, z = 4 * i / n, x = 4 * i % n;
        if (i < Q) cp_async16(ss + z * n + (x ^ (z & 28)), S + ((int64_t)z * n + ky) * n + x);
    }
    cp_async_commit();
    pdl_wait();
    pdl_trigger();
    float4 f[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * T, z = 4 * i / n, x = 4 * i % n;
        if (i < Q) f[k] = *reinterpret_cast<const float4*>(tz + ((int64_t)z * n + ky) * n + x);
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * T, z = 4 * i / n, x = 4 * i % n;
        if (i < Q) *reinterpret_cast<float4*>(s + z * n + (x ^ (z & 28))) = fht_perm4(f[k], z & 3);
    }
    __syncthreads();
    fht_cols<R, false>(t, warp, lane);
    cp_async_wait<0>();
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * T, z = 4 * i / n, x = 4 * i % n;
        if (i < Q) {
            const int e = z * n + (x ^ (z & 28));
            const float4 g = *reinterpret_cast<const float4*>(s + e);
            const float4 w = fht_perm4(*reinterpret_cast<const float4*>(ss + e), z & 3);
            *reinterpret_cast<float4*>(s + e) = make_float4(g.x * w.x, g.y * w.y, g.z * w.z, g.w * w.w);
        }
    }
    __syncthreads();
    fht_cols<R, true>(t, warp, lane);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * T, z = 4 * i / n, x = 4 * i % n;
        if (i < Q)
            *reinterpret_cast<float4*>(tz + ((int64_t)z * n + ky) * n + x) =
                fht_perm4(*reinterpret_cast<const float4*>(s + z * n + (x ^ (z & 28))), z & 3);
    }
}


// ---------------------------------------------------------------- FFT smoothing, n >= 192
// A plane of 192 points or more does not fit in shared memory, so the
// transforms run as five passes over global memory: forward x (row pairs straight from global
// memory, k_fht_rows), forward y (k_fht_cols), forward z + scaling + inverse
// z (k_fht_cols, MODE 1), inverse y, inverse x with per-block sums.  The
// line-pair transform is fht_pair, as above.
constexpr int kFhtBigN = 256;      // the largest power of two the passes serve
constexpr int kFhtRowWarps = 8;     // row pairs per block of k_fht_rows
constexpr int kFhtColThreads = 512; // 16 warps: one column pair each of a 32-column tile

// x transforms of row pairs: warp w of block b takes the kFhtRowPairs row
// pairs starting at rows 2 (kFhtRowPairs (8 b + w) + i), i < kFhtRowPairs,
// of the n^3 array (all z and y), reads them from `in` (all loads first)
// and writes their coefficients to `out` at the same positions.  The pairs
// of a warp are independent chains, so their latencies overlap.  With
// partial, partial[blockIdx.x] gets the compensated sum of the block's
// output and the last block to finish writes their sum (fixed order) to
// *sum_out.
constexpr int kFhtRowPairs = 2;
template <int R, bool INV>
__global__ void __launch_bounds__(32 * kFhtRowWarps, 4)  // four blocks per SM (at most 64 registers)
k_fht_rows(const float* __restrict__ in, float* __restrict__ out, const float2* __restrict__ tw,
           double* __restrict__ partial, unsigned* __restrict__ arrive, double* __restrict__ sum_out) {
    constexpr int n = 32 * R, NP = kFhtRowPairs;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    FhtTw<R> t;
    fht_twiddles<R>(t, tw, lane);  // constant: before the wait
    pdl_wait();
    pdl_trigger();
    const int64_t r0 = 2 * NP * ((int64_t)blockIdx.x * kFhtRowWarps + warp);
    float2 v[NP][R];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const float* a = in + (r0 + 2 * i) * n;
#pragma unroll
        for (int j = 0; j < R; ++j) v[i][j] = make_float2(a[lane + 32 * j], a[n + lane + 32 * j]);
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) fht_pair<R, INV>(v[i], t, lane);
    float acc_s = 0.f, acc_c = 0.f;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        float* o = out + (r0 + 2 * i) * n;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            o[lane + 32 * j] = v[i][j].x;
            o[n + lane + 32 * j] = v[i][j].y;
            if (partial) {
                two_sum_add(acc_s, acc_c, v[i][j].x);
                two_sum_add(acc_s, acc_c, v[i][j].y);
            }
        }
    }
    if (partial) sum_last_block((double)acc_s + (double)acc_c, partial, arrive, sum_out);
}

// Transforms along an axis of element stride ls (y: n, z: n^2) for the 32
// consecutive x of tile blockIdx.x, at offset blockIdx.y * os of the other
// axis (y lines: z planes, os = n^2; z lines: y rows, os = n).  The n x 32
// tile sits in shared memory with element (p, c) at 32 p + (c ^ (p mod 32))
// (16-byte groups kept together, so rows load as float4 and both rows and
// columns are free of bank conflicts); one warp per column pair.  MODE 0: a
// forward (INV false) or inverse transform, in place.  MODE 1: forward,
// scaling by S (laid out like the data; its tile copied in by cp.async
// meanwhile), inverse.
template <int R, int MODE, bool INV>
__global__ void __launch_bounds__(kFhtColThreads, 2)  // two blocks per SM (at most 64 registers)
k_fht_cols(float* __restrict__ d, int64_t ls, int64_t os, const float2* __restrict__ tw,
           const float* __restrict__ S) {
    constexpr int n = 32 * R, Q = n * 32 / 4, PER = Q / kFhtColThreads;
    static_assert(PER * kFhtColThreads == Q, "float4 groups per thread");
    extern __shared__ __align__(16) unsigned char fht_smem[];
    float* s = reinterpret_cast<float*>(fht_smem);
    float* ss = s + n * 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.y * os + (int64_t)blockIdx.x * 32;
    FhtTw<R> t;
    fht_twiddles<R>(t, tw, lane);
    if constexpr (MODE == 1) {
#pragma unroll
        for (int k = 0; k < PER; ++k) {  // S is constant: before the wait
            const int i = tid + k * kFhtColThreads, p = i >> 3, c = (i & 7) * 4;
            cp_async16(ss + 32 * p + (c ^ (p & 28)), S + base + p * ls + c);
        }
        cp_async_commit();
    }
    pdl_wait();
    pdl_trigger();
    float4 f[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * kFhtColThreads, p = i >> 3, c = (i & 7) * 4;
        f[k] = *reinterpret_cast<const float4*>(d + base + p * ls + c);
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * kFhtColThreads, p = i >> 3, c = (i & 7) * 4;
        *reinterpret_cast<float4*>(s + 32 * p + (c ^ (p & 28))) = fht_perm4(f[k], p & 3);
    }
    __syncthreads();
    const int c0 = 2 * warp;  // this warp's column pair
    const unsigned a = 4u * (unsigned)(32 * lane + (c0 ^ lane)), b = 4u * (unsigned)(32 * lane + ((c0 + 1) ^ lane));
    constexpr unsigned JS = 4u * 32u * 32u;
    if constexpr (MODE == 0) {
        warp_fht2<R, INV, JS>(a, b, a, b, t, lane);
    } else {
        warp_fht2<R, false, JS>(a, b, a, b, t, lane);
        cp_async_wait<0>();
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = tid + k * kFhtColThreads, p = i >> 3, c = (i & 7) * 4;
            const int e = 32 * p + (c ^ (p & 28));
            const float4 g = *reinterpret_cast<const float4*>(s + e);
            const float4 w = fht_perm4(*reinterpret_cast<const float4*>(ss + e), p & 3);
            *reinterpret_cast<float4*>(s + e) = make_float4(g.x * w.x, g.y * w.y, g.z * w.z, g.w * w.w);
        }
        __syncthreads();
        warp_fht2<R, true, JS>(a, b, a, b, t, lane);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = tid + k * kFhtColThreads, p = i >> 3, c = (i & 7) * 4;
        *reinterpret_cast<float4*>(d + base + p * ls + c) =
            fht_perm4(*reinterpret_cast<const float4*>(s + 32 * p + (c ^ (p & 28))), p & 3);
    }
}

// Shared memory of k_fht_cols: the tile, and in MODE 1 the tile of S.
inline size_t fht_cols_smem_bytes(int n, int mode) { return (size_t)(mode ? 2 : 1) * n * 32 * sizeof(float); }

// Meshes the FFT smoothing handles: a plane per block up to 128, five
// passes over global memory at 192, 256, 320 and 384 (192 = 3 x 64, 320 =
// 5 x 64, 384 = 3 x 128 by the mixed-radix transform).
inline bool fht_passes(int n) { return n == 192 || n == kFhtBigN || n == 320 || n == 384; }
inline bool fht_supported(int n) { return n == 32 || n == 64 || n == kFhtMaxN || fht_passes(n); }
// Radix-3/5 factor of a supported length (1 for powers of two).
inline int fht_q(int n) { return n % 3 == 0 ? 3 : n % 5 == 0 ? 5 : 1; }

// ---------------------------------------------------------------- interpolation
// F_a = -ke Q_a sum_n W(r_a - r_n) (D phi)_n with central differences
// (Eq. 21), one thread per particle in cell order; writes the total force
// (adding the short-range part) and the two parts in original order.  R is
// the arithmetic type of the weights, differences and the 64-term sums (FP64,
// or FP32 from an FP32 copy of phi in mixed mode); the result is FP64.
template <typename R>
__global__ void __launch_bounds__(P3_THREADS)
k_gather(int np, const PQ* __restrict__ xq, const int* __restrict__ order, int n, double inv_h,
         double ke, const R* __restrict__ phi, const double* __restrict__ Fsr_s,
         double* __restrict__ F, double* __restrict__ Flr, double* __restrict__ Fsr) {
    pdl_wait();
    pdl_trigger();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const PQ p = xq[s];
    double wxd[4], wyd[4], wzd[4];
    const int bx = bspline_axis(p.x, inv_h, n, wxd);
    const int by = bspline_axis(p.y, inv_h, n, wyd);
    const int bz = bspline_axis(p.z, inv_h, n, wzd);
    R wx[4], wy[4], wz[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        wx[k] = (R)wxd[k];
        wy[k] = (R)wyd[k];
        wz[k] = (R)wzd[k];
    }
    int ix[4], ixm[4], ixp[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        ix[a] = wrap_idx(bx + a, n);
        ixm[a] = ix[a] == 0 ? n - 1 : ix[a] - 1;
        ixp[a] = ix[a] == n - 1 ? 0 : ix[a] + 1;
    }
    R gx = 0, gy = 0, gz = 0;
    for (int c = 0; c < 4; ++c) {
        const int iz = wrap_idx(bz + c, n);
        const int izm = iz == 0 ? n - 1 : iz - 1, izp = iz == n - 1 ? 0 : iz + 1;
        for (int b = 0; b < 4; ++b) {
            const int iy = wrap_idx(by + b, n);
            const int iym = iy == 0 ? n - 1 : iy - 1, iyp = iy == n - 1 ? 0 : iy + 1;
            const R wyz = wy[b] * wz[c];
            const R* row = phi + ((int64_t)iz * n + iy) * n;
            const R* rym = phi + ((int64_t)iz * n + iym) * n;
            const R* ryp = phi + ((int64_t)iz * n + iyp) * n;
            const R* rzm = phi + ((int64_t)izm * n + iy) * n;
            const R* rzp = phi + ((int64_t)izp * n + iy) * n;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const R w = wyz * wx[a];
                gx += w * (row[ixp[a]] - row[ixm[a]]);
                gy += w * (ryp[ix[a]] - rym[ix[a]]);
                gz += w * (rzp[ix[a]] - rzm[ix[a]]);
            }
        }
    }
    const double scale = -ke * p.w * 0.5 * inv_h;
    const int i = order[s];
    const double f[3] = {scale * (double)gx, scale * (double)gy, scale * (double)gz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double sr = Fsr_s[3 * s + d];
        F[3 * i + d] = sr + f[d];
        Flr[3 * i + d] = f[d];
        Fsr[3 * i + d] = sr;
    }
}

// FP32 interpolation (Eq. 21) from precomputed mesh coordinates and the FP32
// copy of phi, one thread per particle.  The central-difference sum is
// regrouped by summation by parts, term for term over the stencil positions
// (so it holds with periodic wrap on any mesh):
//   sum_n W_n (phi_{n+1} - phi_{n-1}) = sum_m phi_m (W_{m-1} - W_{m+1}),
// per axis, with the weights zero outside the 4-point support.  The x
// gradient then needs phi on the 6x4x4 block around the stencil, y on 4x6x4
// and z on 4x4x6: 160 distinct loads instead of 64 x 6.  Output as k_gather.
static __global__ void __launch_bounds__(P3_THREADS)
k_gather_mp(int np, const MeshPt* __restrict__ mp, const int* __restrict__ order, int n, double inv_h,
            double ke, const float* __restrict__ phi, const double* __restrict__ Fsr_s,
            double* __restrict__ F, double* __restrict__ Flr, double* __restrict__ Fsr,
            const double* __restrict__ hdt_acc, double* __restrict__ v) {
    pdl_wait();
    pdl_trigger();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const MeshPt p = mp[s];
    // e: weights at stencil positions -1..4 (zero at -1 and 4); d: W_{m-1} - W_{m+1}
    float ex[6], ey[6], ez[6], dx[6], dy[6], dz[6];
    {
        float w[4];
        bspline4f(p.tx, w);
        ex[0] = 0.0f; ex[1] = w[0]; ex[2] = w[1]; ex[3] = w[2]; ex[4] = w[3]; ex[5] = 0.0f;
        bspline4f(p.ty, w);
        ey[0] = 0.0f; ey[1] = w[0]; ey[2] = w[1]; ey[3] = w[2]; ey[4] = w[3]; ey[5] = 0.0f;
        bspline4f(p.tz, w);
        ez[0] = 0.0f; ez[1] = w[0]; ez[2] = w[1]; ez[3] = w[2]; ez[4] = w[3]; ez[5] = 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        dx[j] = (j > 0 ? ex[j - 1] : 0.0f) - (j < 5 ? ex[j + 1] : 0.0f);
        dy[j] = (j > 0 ? ey[j - 1] : 0.0f) - (j < 5 ? ey[j + 1] : 0.0f);
        dz[j] = (j > 0 ? ez[j - 1] : 0.0f) - (j < 5 ? ez[j + 1] : 0.0f);
    }
    int ix[6], iy[6], iz[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        ix[j] = wrap_idx(p.bx - 1 + j, n);
        iy[j] = wrap_idx(p.by - 1 + j, n);
        iz[j] = wrap_idx(p.bz - 1 + j, n);
    }
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const bool zin = c >= 1 && c <= 4;
#pragma unroll
        for (int b = 0; b < 6; ++b) {
            const bool yin = b >= 1 && b <= 4;
            if (!zin && !yin) continue;
            const float* row = phi + ((int64_t)iz[c] * n + iy[b]) * n;
            if (zin && yin) {
                const float wyz = ey[b] * ez[c], dyz = dy[b] * ez[c], ydz = ey[b] * dz[c];
#pragma unroll
                for (int a = 0; a < 6; ++a) {
                    const float v = row[ix[a]];
                    gx += dx[a] * wyz * v;
                    if (a >= 1 && a <= 4) {
                        const float xv = ex[a] * v;
                        gy += dyz * xv;
                        gz += ydz * xv;
                    }
                }
            } else if (zin) {  // rows y = -1 and 4: y gradient only
                const float dyz = dy[b] * ez[c];
#pragma unroll
                for (int a = 1; a <= 4; ++a) gy += dyz * ex[a] * row[ix[a]];
            } else {           // planes z = -1 and 4: z gradient only
                const float ydz = ey[b] * dz[c];
#pragma unroll
                for (int a = 1; a <= 4; ++a) gz += ydz * ex[a] * row[ix[a]];
            }
        }
    }
    // g = sum_m phi_m (W_{m-1} - W_{m+1}) = sum_n W_n (phi_{n+1} - phi_{n-1});
    // F = -ke Q g / (2h)
    const double scale = -ke * (double)p.q * 0.5 * inv_h;
    const int i = order[s];
    const double f[3] = {scale * (double)gx, scale * (double)gy, scale * (double)gz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double sr = Fsr_s[3 * s + d];
        const double Ft = sr + f[d];
        F[3 * i + d] = Ft;
        Flr[3 * i + d] = f[d];
        Fsr[3 * i + d] = sr;
        // the closing half kick of the step (k_kick's arithmetic), when no
        // other term is added to F after this kernel
        if (v != nullptr) v[3 * i + d] += hdt_acc[i] * Ft;
    }
}

// Analytic-gradient interpolation (an option; the paper's force is the
// finite-difference one above): F_a = -ke Q_a sum_n grad W(r_a - r_n) phi_n,
// grad W = inv_h (w'(tx) w(ty) w(tz), ...), the exact gradient of
// V_LR = 1/2 ke phi^T q for phi = G q with G symmetric, so the long-range
// force conserves energy (but is not exactly antisymmetric: momentum is
// conserved only to the discretisation error).  64 loads of phi per particle.
// FP32 from the mesh coordinates and the FP32 phi copy; the constant offset of
// that copy drops out (the derivative weights sum to zero).
static __global__ void __launch_bounds__(P3_THREADS)
k_gather_grad_mp(int np, const MeshPt* __restrict__ mp, const int* __restrict__ order, int n, double inv_h,
                 double ke, const float* __restrict__ phi, const double* __restrict__ Fsr_s,
                 double* __restrict__ F, double* __restrict__ Flr, double* __restrict__ Fsr) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const MeshPt p = mp[s];
    float wx[4], wy[4], wz[4], dx[4], dy[4], dz[4];
    bspline4f(p.tx, wx);
    bspline4f(p.ty, wy);
    bspline4f(p.tz, wz);
    bspline4f_deriv(p.tx, dx);
    bspline4f_deriv(p.ty, dy);
    bspline4f_deriv(p.tz, dz);
    int ix[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) ix[a] = wrap_idx(p.bx + a, n);
    float gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int iz = wrap_idx(p.bz + c, n);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int iy = wrap_idx(p.by + b, n);
            const float* row = phi + ((int64_t)iz * n + iy) * n;
            const float wyz = wy[b] * wz[c], dyz = dy[b] * wz[c], ydz = wy[b] * dz[c];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float v = row[ix[a]];
                gx += dx[a] * wyz * v;
                gy += wx[a] * dyz * v;
                gz += wx[a] * ydz * v;
            }
        }
    }
    const double scale = -ke * (double)p.q * inv_h;
    const int i = order[s];
    const double f[3] = {scale * (double)gx, scale * (double)gy, scale * (double)gz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double sr = Fsr_s[3 * s + d];
        F[3 * i + d] = sr + f[d];
        Flr[3 * i + d] = f[d];
        Fsr[3 * i + d] = sr;
    }
}

// The same in FP64 from the cell-ordered positions and the FP64 phi.
static __global__ void __launch_bounds__(P3_THREADS)
k_gather_grad64(int np, const PQ* __restrict__ xq, const int* __restrict__ order, int n, double inv_h, double ke,
                const double* __restrict__ phi, const double* __restrict__ Fsr_s, double* __restrict__ F,
                double* __restrict__ Flr, double* __restrict__ Fsr) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const PQ p = xq[s];
    double w[3][4], d[3][4];
    int base[3];
    const double xs[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        double u = xs[ax] * inv_h;
        if (!(u >= 0.0 && u <= (double)n)) u = 0.0;
        const double fl = floor(u);
        bspline4(u - fl, w[ax]);
        bspline4_deriv(u - fl, d[ax]);
        base[ax] = wrap_idx((int)fl - 1, n);
    }
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int c = 0; c < 4; ++c) {
        const int iz = wrap_idx(base[2] + c, n);
        for (int b = 0; b < 4; ++b) {
            const int iy = wrap_idx(base[1] + b, n);
            const double* row = phi + ((int64_t)iz * n + iy) * n;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const double v = row[wrap_idx(base[0] + a, n)];
                gx += d[0][a] * w[1][b] * w[2][c] * v;
                gy += w[0][a] * d[1][b] * w[2][c] * v;
                gz += w[0][a] * w[1][b] * d[2][c] * v;
            }
        }
    }
    const double scale = -ke * p.w * inv_h;
    const int i = order[s];
    const double f[3] = {scale * gx, scale * gy, scale * gz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double sr = Fsr_s[3 * s + k];
        F[3 * i + k] = sr + f[k];
        Flr[3 * i + k] = f[k];
        Fsr[3 * i + k] = sr;
    }
}

}  // namespace p3
