// Particle-side kernels: velocity-Verlet updates, the cell list and the
// short-range pair forces.
#pragma once

#include "common.cuh"

namespace p3 {

// Velocity-Verlet half kick (Sec. 2; supporting information Sec. 1):
// v += (dt/2) F / m.  hdt_acc[i] = 0.5 dt ACCEL / m_i.
__global__ void k_kick(int n, double* __restrict__ v, const double* __restrict__ F,
                       const double* __restrict__ hdt_acc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = hdt_acc[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) v[3 * i + d] += a * F[3 * i + d];
}

__device__ __forceinline__ double wrap_pos(double x, double L) {
    x = x - L * floor(x / L);
    if (x < 0.0) x += L;
    if (x >= L) x = 0.0;
    return x;
}

// Half kick, drift r += dt v, and wrap into [0, L).
__global__ void k_kick_drift(int n, double* __restrict__ r, double* __restrict__ v,
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

__global__ void k_wrap(int n, double* __restrict__ r, double L) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    r[i] = wrap_pos(r[i], L);
}

// ---------------------------------------------------------------- cell list
// Cell of each particle, c = min(floor(r * nc/L), nc-1) per axis, x fastest,
// and per-cell counts.
__global__ void k_cell_count(int n, const double* __restrict__ r, double inv_cell, int nc,
                             int* __restrict__ cell, int* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int cx = min((int)floor(r[3 * i + 0] * inv_cell), nc - 1);
    const int cy = min((int)floor(r[3 * i + 1] * inv_cell), nc - 1);
    const int cz = min((int)floor(r[3 * i + 2] * inv_cell), nc - 1);
    const int c = (cz * nc + cy) * nc + cx;
    cell[i] = c;
    atomicAdd(&count[c], 1);
}

// Exclusive scan of m counts into start[0..m] with one block of 1024 threads;
// also clears the per-cell fill counters.
__global__ void __launch_bounds__(1024) k_scan_cells(int m, const int* __restrict__ count,
                                                     int* __restrict__ start, int* __restrict__ fill) {
    __shared__ int warp_tot[32];
    const int tid = threadIdx.x;
    const int chunk = (m + blockDim.x - 1) / blockDim.x;
    const int beg = min(tid * chunk, m), end = min(beg + chunk, m);
    int local = 0;
    for (int j = beg; j < end; ++j) local += count[j];
    // inclusive warp scan
    int v = local;
    const int lane = tid & 31, wid = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int w = warp_tot[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    int run = v - local + (wid > 0 ? warp_tot[wid - 1] : 0);
    for (int j = beg; j < end; ++j) {
        start[j] = run;
        fill[j] = 0;
        run += count[j];
    }
    if (tid == blockDim.x - 1) start[m] = warp_tot[31];
}

__global__ void k_cell_scatter(int n, const int* __restrict__ cell, const int* __restrict__ start,
                               int* __restrict__ fill, int* __restrict__ order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell[i];
    order[start[c] + atomicAdd(&fill[c], 1)] = i;
}

// Sort each cell's members by particle index so the order is deterministic.
__global__ void k_cell_sort(int m, const int* __restrict__ start, int* __restrict__ order) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
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

// Gather particle data into cell order: xq = (x, y, z, Q) and the
// cell-local coordinates x - c l (FP64 and FP32 copies) used by the pair kernel.
__global__ void k_gather_sorted(int n, const int* __restrict__ order, const double* __restrict__ r,
                                const double* __restrict__ Q, const int* __restrict__ type,
                                const int* __restrict__ mol, const int* __restrict__ cell, int nc,
                                double lcell, PQ* __restrict__ xq, PQ* __restrict__ xl64,
                                float4* __restrict__ xl32, int* __restrict__ ts, int* __restrict__ ms,
                                int* __restrict__ cs) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int i = order[s];
    const int c = cell[i];
    const double x = r[3 * i], y = r[3 * i + 1], z = r[3 * i + 2], q = Q[i];
    xq[s] = PQ{x, y, z, q};
    const double lx = x - (c % nc) * lcell, ly = y - ((c / nc) % nc) * lcell, lz = z - (c / (nc * nc)) * lcell;
    xl64[s] = PQ{lx, ly, lz, q};
    xl32[s] = make_float4((float)lx, (float)ly, (float)lz, (float)q);
    ts[s] = type ? type[i] : 0;
    ms[s] = mol ? mol[i] : -1;
    cs[s] = c;
}

// ---------------------------------------------------------------- pair forces
struct SRTable {
    int kind;      // 0 none, 1 BMH, 2 LJ
    int nt;
    double p[5][16];
};

// Per-pair screened Coulomb (Eq. 19 with alpha = 1/(sqrt2 sigma); energy
// Eq. 5) and the non-Coulomb term.  Returns F/r scaled by ke for the Coulomb
// part; energies are accumulated unscaled.
template <int KIND, typename R>
__device__ __forceinline__ R pair_terms(R r2, R qq, R alpha, const SRTable& tab, int k, R& ec, R& ev,
                                        R& fvdw) {
    const R ir = (R)1 / sqrt(r2);
    const R rr = r2 * ir;
    const R ar = alpha * rr;
    const R erfcv = erfc(ar);
    const R ex = exp(-ar * ar);
    const R ir2 = ir * ir;
    ec = qq * erfcv * ir;
    ev = (R)0;
    fvdw = (R)0;
    if (KIND == 1) {
        const R A = (R)tab.p[0][k], rho = (R)tab.p[1][k], sg = (R)tab.p[2][k];
        const R C = (R)tab.p[3][k], D = (R)tab.p[4][k];
        const R eb = A * exp((sg - rr) / rho);
        const R ir6 = ir2 * ir2 * ir2, ir8 = ir6 * ir2;
        ev = eb - C * ir6 - D * ir8;
        fvdw = (eb / rho - (R)6 * C * ir6 * ir - (R)8 * D * ir8 * ir) * ir;
    } else if (KIND == 2) {
        const R eps = (R)tab.p[0][k];
        if (eps != (R)0) {
            const R sg = (R)tab.p[1][k];
            const R sr2 = sg * sg * ir2;
            const R sr6 = sr2 * sr2 * sr2;
            ev = (R)4 * eps * (sr6 * sr6 - sr6);
            fvdw = (R)24 * eps * ((R)2 * sr6 * sr6 - sr6) * ir2;
        }
    }
    return qq * (erfcv * ir + (R)kTwoOverSqrtPi * alpha * ex) * ir2;
}

// Short-range forces on particle s (cell order) from every particle image
// within r_cut, found in the 5x5x5 block of cells of edge l >= r_cut/2 around
// it: Eq. 19 plus the Born-Mayer or Lennard-Jones term.  One warp per
// particle, each lane walking a share of the 125 neighbour cells; a
// particle's neighbour j in unwrapped cell c_i + d sits at the image
// (c_i + d) l + x_j,loc, so the separation is x_i,loc - x_j,loc - d l with no
// periodic shift.  Pairs within one molecule closer than L/2 (the nearest
// image) are excluded.  Writes the force and half of the pair energies of s;
// no atomics.  R is the arithmetic type (double, or float in mixed mode with
// FP32 cell-local coordinates and FP64 accumulation across lanes).
template <int KIND, typename R, typename LQ>
__global__ void __launch_bounds__(P3_THREADS)
k_pair(int n, const LQ* __restrict__ xl, const int* __restrict__ ts, const int* __restrict__ ms,
       const int* __restrict__ cs, const int* __restrict__ start, int nc, double lcell, double rc2,
       double halfL2, double alpha, double ke, SRTable tab, double* __restrict__ Fs,
       double* __restrict__ ecs, double* __restrict__ evs) {
    const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (s >= n) return;
    const LQ pi = xl[s];
    const int ti = ts[s];
    const int mi = ms[s];
    const int ci = cs[s];
    const int cx = ci % nc, cy = (ci / nc) % nc, cz = ci / (nc * nc);
    const R lc = (R)lcell, r2c = (R)rc2, hl2 = (R)halfL2, al = (R)alpha;
    R fx = 0, fy = 0, fz = 0, ec = 0, ev = 0;
    for (int o = lane; o < 125; o += 32) {
        const int dx = o % 5 - 2, dy = (o / 5) % 5 - 2, dz = o / 25 - 2;
        int xx = cx + dx, yy = cy + dy, zz = cz + dz;
        while (xx < 0) xx += nc;
        while (xx >= nc) xx -= nc;
        while (yy < 0) yy += nc;
        while (yy >= nc) yy -= nc;
        while (zz < 0) zz += nc;
        while (zz >= nc) zz -= nc;
        const bool home = dx == 0 && dy == 0 && dz == 0;
        const R ox = (R)dx * lc, oy = (R)dy * lc, oz = (R)dz * lc;
        const int c = (zz * nc + yy) * nc + xx;
        const int e = start[c + 1];
        for (int t = start[c]; t < e; ++t) {
            if (home && t == s) continue;
            const LQ pj = xl[t];
            const R ddx = (R)pi.x - (R)pj.x - ox;
            const R ddy = (R)pi.y - (R)pj.y - oy;
            const R ddz = (R)pi.z - (R)pj.z - oz;
            const R r2 = ddx * ddx + ddy * ddy + ddz * ddz;
            if (r2 >= r2c) continue;
            if (mi >= 0 && ms[t] == mi && r2 < hl2) continue;
            R e_c, e_v, f_v;
            const R fr = pair_terms<KIND, R>(r2, (R)pi.w * (R)pj.w, al, tab, ti * tab.nt + ts[t], e_c, e_v, f_v);
            const R f = (R)ke * fr + f_v;
            fx += f * ddx;
            fy += f * ddy;
            fz += f * ddz;
            ec += e_c;
            ev += e_v;
        }
    }
    double dfx = fx, dfy = fy, dfz = fz, dec = ec, dev = ev;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        dfx += __shfl_xor_sync(0xffffffffu, dfx, w);
        dfy += __shfl_xor_sync(0xffffffffu, dfy, w);
        dfz += __shfl_xor_sync(0xffffffffu, dfz, w);
        dec += __shfl_xor_sync(0xffffffffu, dec, w);
        dev += __shfl_xor_sync(0xffffffffu, dev, w);
    }
    if (lane == 0) {
        Fs[3 * s + 0] = dfx;
        Fs[3 * s + 1] = dfy;
        Fs[3 * s + 2] = dfz;
        ecs[s] = 0.5 * ke * dec;
        evs[s] = 0.5 * dev;
    }
}

// SPC/Fw intramolecular terms, one thread per (h1, o, h2) molecule: harmonic
// bonds and angle (Table S1) and the subtraction of the mesh part
// ke QQ erf(r/(sqrt2 sigma))/r of the three intramolecular pairs.  Adds into
// F (original order) and writes the bonded force and energies.
__global__ void k_water(int nmol, const int* __restrict__ tri, const double* __restrict__ r,
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
