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

// Gather particle data into cell order: xq = (x, y, z, Q).
__global__ void k_gather_sorted(int n, const int* __restrict__ order, const double* __restrict__ r,
                                const double* __restrict__ Q, const int* __restrict__ type,
                                const int* __restrict__ mol, const int* __restrict__ cell,
                                PQ* __restrict__ xq, int* __restrict__ ts, int* __restrict__ ms,
                                int* __restrict__ cs) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int i = order[s];
    xq[s] = PQ{r[3 * i], r[3 * i + 1], r[3 * i + 2], Q[i]};
    ts[s] = type ? type[i] : 0;
    ms[s] = mol ? mol[i] : -1;
    cs[s] = cell[i];
}

// ---------------------------------------------------------------- pair forces
struct SRTable {
    int kind;      // 0 none, 1 BMH, 2 LJ
    int nt;
    double p[5][16];
};

// Short-range forces on particle s (cell order) from every particle image
// within r_cut, found in the 5x5x5 block of cells of edge >= r_cut/2 around
// it: the erfc-screened Coulomb force of Eq. 19 (written with alpha =
// 1/(sqrt2 sigma)) plus the Born-Mayer or Lennard-Jones term.  Pairs within
// one molecule at separation below L/2 (the nearest image) are excluded.
// Writes per-particle force and half of its pair energies; no atomics.
// MIXED evaluates the pair functions in FP32 from an FP64 separation and
// accumulates in FP64.
template <int KIND, bool MIXED>
__global__ void __launch_bounds__(P3_THREADS)
k_pair(int n, const PQ* __restrict__ xq, const int* __restrict__ ts, const int* __restrict__ ms,
       const int* __restrict__ cs, const int* __restrict__ start, int nc, double L, double rc2,
       double halfL2, double alpha, double ke, SRTable tab, double* __restrict__ Fs,
       double* __restrict__ ecs, double* __restrict__ evs) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const PQ pi = xq[s];
    const int ti = ts[s];
    const int mi = ms[s];
    const int ci = cs[s];
    const int cx = ci % nc, cy = (ci / nc) % nc, cz = ci / (nc * nc);
    double fx = 0.0, fy = 0.0, fz = 0.0, ec = 0.0, ev = 0.0;
    for (int dz = -2; dz <= 2; ++dz) {
        int zz = cz + dz, kz = 0;
        while (zz < 0) { zz += nc; --kz; }
        while (zz >= nc) { zz -= nc; ++kz; }
        for (int dy = -2; dy <= 2; ++dy) {
            int yy = cy + dy, ky = 0;
            while (yy < 0) { yy += nc; --ky; }
            while (yy >= nc) { yy -= nc; ++ky; }
            for (int dx = -2; dx <= 2; ++dx) {
                int xx = cx + dx, kx = 0;
                while (xx < 0) { xx += nc; --kx; }
                while (xx >= nc) { xx -= nc; ++kx; }
                const bool home = (kx | ky | kz) == 0;
                const double sx = kx * L, sy = ky * L, sz = kz * L;
                const int c = (zz * nc + yy) * nc + xx;
                const int e = start[c + 1];
                for (int t = start[c]; t < e; ++t) {
                    if (home && t == s) continue;
                    const PQ pj = xq[t];
                    const double ddx = pi.x - (pj.x + sx);
                    const double ddy = pi.y - (pj.y + sy);
                    const double ddz = pi.z - (pj.z + sz);
                    const double r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                    if (r2 >= rc2) continue;
                    if (mi >= 0 && ms[t] == mi && r2 < halfL2) continue;
                    const double qq = pi.w * pj.w;
                    double fr, e_c, e_v = 0.0, f_v = 0.0;
                    if (MIXED) {
                        const float r2f = (float)r2;
                        const float ir = rsqrtf(r2f);
                        const float rr = r2f * ir;
                        const float ar = (float)alpha * rr;
                        const float erfcv = erfcf(ar);
                        const float ex = expf(-ar * ar);
                        const float ir2 = ir * ir;
                        e_c = (double)((float)qq * erfcv * ir);
                        fr = (double)((float)qq * (erfcv * ir + (float)(kTwoOverSqrtPi * alpha) * ex) * ir2);
                        if (KIND == 1) {
                            const int k = ti * tab.nt + ts[t];
                            const float A = (float)tab.p[0][k], rho = (float)tab.p[1][k], sg = (float)tab.p[2][k];
                            const float C = (float)tab.p[3][k], D = (float)tab.p[4][k];
                            const float eb = A * expf((sg - rr) / rho);
                            const float ir6 = ir2 * ir2 * ir2, ir8 = ir6 * ir2;
                            e_v = (double)(eb - C * ir6 - D * ir8);
                            f_v = (double)((eb / rho - 6.0f * C * ir6 * ir - 8.0f * D * ir8 * ir) * ir);
                        } else if (KIND == 2) {
                            const int k = ti * tab.nt + ts[t];
                            const float eps = (float)tab.p[0][k];
                            if (eps != 0.0f) {
                                const float sg = (float)tab.p[1][k];
                                const float sr2 = sg * sg * ir2;
                                const float sr6 = sr2 * sr2 * sr2;
                                e_v = (double)(4.0f * eps * (sr6 * sr6 - sr6));
                                f_v = (double)(24.0f * eps * (2.0f * sr6 * sr6 - sr6) * ir2);
                            }
                        }
                    } else {
                        const double rr = sqrt(r2);
                        const double ir = 1.0 / rr;
                        const double ar = alpha * rr;
                        const double erfcv = erfc(ar);
                        const double ex = exp(-ar * ar);
                        const double ir2 = ir * ir;
                        e_c = qq * erfcv * ir;
                        fr = qq * (erfcv * ir + kTwoOverSqrtPi * alpha * ex) * ir2;
                        if (KIND == 1) {
                            const int k = ti * tab.nt + ts[t];
                            const double rho = tab.p[1][k];
                            const double eb = tab.p[0][k] * exp((tab.p[2][k] - rr) / rho);
                            const double ir6 = ir2 * ir2 * ir2, ir8 = ir6 * ir2;
                            e_v = eb - tab.p[3][k] * ir6 - tab.p[4][k] * ir8;
                            f_v = (eb / rho - 6.0 * tab.p[3][k] * ir6 * ir - 8.0 * tab.p[4][k] * ir8 * ir) * ir;
                        } else if (KIND == 2) {
                            const int k = ti * tab.nt + ts[t];
                            const double eps = tab.p[0][k];
                            if (eps != 0.0) {
                                const double sg = tab.p[1][k];
                                const double sr2 = sg * sg * ir2;
                                const double sr6 = sr2 * sr2 * sr2;
                                e_v = 4.0 * eps * (sr6 * sr6 - sr6);
                                f_v = 24.0 * eps * (2.0 * sr6 * sr6 - sr6) * ir2;
                            }
                        }
                    }
                    const double f = ke * fr + f_v;
                    fx += f * ddx;
                    fy += f * ddy;
                    fz += f * ddz;
                    ec += e_c;
                    ev += e_v;
                }
            }
        }
    }
    Fs[3 * s + 0] = fx;
    Fs[3 * s + 1] = fy;
    Fs[3 * s + 2] = fz;
    ecs[s] = 0.5 * ke * ec;
    evs[s] = 0.5 * ev;
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
