// Mesh-side kernels: charge assignment, diffusion smoothing, reductions, the
// Mass-Zero prediction / constraint residual / field update, the multigrid
// operators, and the force interpolation.  Mesh arrays are N^3, x fastest:
// index (iz*N + iy)*N + ix.  T is the bulk mesh type (double or float).
#pragma once

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

__device__ __forceinline__ void unflatten(int64_t i, int n, int& x, int& y, int& z) {
    x = (int)(i % n);
    const int64_t r = i / n;
    y = (int)(r % n);
    z = (int)(r / n);
}

// ---------------------------------------------------------------- assignment
// q_n += Q_a W(u_a - n): cubic B-spline charge assignment (Sec. 2), one thread
// per particle in cell order, 64 atomic adds.
template <typename T>
__global__ void __launch_bounds__(P3_THREADS)
k_spread(int np, const PQ* __restrict__ xq, int n, double inv_h, T* __restrict__ q) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const PQ p = xq[s];
    double wx[4], wy[4], wz[4];
    const int bx = bspline_axis(p.x, inv_h, n, wx);
    const int by = bspline_axis(p.y, inv_h, n, wy);
    const int bz = bspline_axis(p.z, inv_h, n, wz);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int iz = wrap_idx(bz + c, n);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int iy = wrap_idx(by + b, n);
            const double wyz = p.w * wy[b] * wz[c];
            T* row = q + ((int64_t)iz * n + iy) * n;
#pragma unroll
            for (int a = 0; a < 4; ++a) atomicAdd(row + wrap_idx(bx + a, n), (T)(wyz * wx[a]));
        }
    }
}

// ---------------------------------------------------------------- smoothing
// One explicit diffusion step out = in + c M in (reading of Sec. 2's
// diffusion-based smoothing).
template <typename T>
__global__ void __launch_bounds__(P3_THREADS)
k_diffuse(int n, const T* __restrict__ in, T* __restrict__ out, T c) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * n * n) return;
    int x, y, z;
    unflatten(i, n, x, y, z);
    const T v = in[i];
    out[i] = v + c * (nb6(in, x, y, z, n) - (T)6 * v);
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
__global__ void k_mv2_partial(int np, const double* __restrict__ v, const double* __restrict__ m,
                              double* __restrict__ partial) {
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x)
        acc += m[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
    acc = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// Sum of nb partials (in a fixed order) into out[0].
__global__ void k_sum_final(int nb, const double* __restrict__ partial, double* __restrict__ out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) out[0] = acc;
}

// ---------------------------------------------------------------- Mass-Zero
// Predicted constraint residual (Eq. 17) with the gauge fix:
//   sigma_p = (h/4pi) M (2 phi^k - phi^{k-1}) + q^s - mean(q^s)
// and the multiplier guess y0 (Sec. 3.3): order 0 -> 0, 1 -> y^k,
// 2 -> 2y^k - y^{k-1}, 3 -> 3y^k - 3y^{k-1} + y^{k-2}.
template <typename T>
__global__ void __launch_bounds__(P3_THREADS)
k_predict(int n, const double* __restrict__ phik, const double* __restrict__ phikm1,
          const T* __restrict__ qs, const double* __restrict__ qsum, double inv_pts, double hc,
          const double* __restrict__ y1, const double* __restrict__ y2, const double* __restrict__ y3,
          int order, double* __restrict__ sig, double* __restrict__ y0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * n * n) return;
    int x, y, z;
    unflatten(i, n, x, y, z);
    const double mk = nb6(phik, x, y, z, n) - 6.0 * phik[i];
    const double mkm1 = nb6(phikm1, x, y, z, n) - 6.0 * phikm1[i];
    const double mean = qsum[0] * inv_pts;
    sig[i] = hc * (2.0 * mk - mkm1) + ((double)qs[i] - mean);
    double g = 0.0;
    if (order == 1) g = y1[i];
    else if (order == 2) g = 2.0 * y1[i] - y2[i];
    else if (order == 3) g = 3.0 * y1[i] - 3.0 * y2[i] + y3[i];
    y0[i] = g;
}

// Fine-level FP64 residual r = sigma_p - M y, stored in the bulk type for the
// correction V-cycle, and max_n |r_n| (Eq. 20) folded into *rmax with an
// atomic max on the bit pattern (non-negative doubles order like integers).
// A NaN or Inf residual is recorded as +Inf.
template <typename T>
__global__ void __launch_bounds__(P3_THREADS)
k_resid_fine(int n, const double* __restrict__ yv, const double* __restrict__ sig, T* __restrict__ r,
             unsigned long long* __restrict__ rmax) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0.0;
    if (i < (int64_t)n * n * n) {
        int x, y, z;
        unflatten(i, n, x, y, z);
        const double res = sig[i] - (nb6(yv, x, y, z, n) - 6.0 * yv[i]);
        r[i] = (T)res;
        a = fabs(res);
        if (!(a <= 1.0e308)) a = __longlong_as_double(0x7ff0000000000000LL);
    }
    a = block_max(a);
    if (threadIdx.x == 0) atomicMax(rmax, (unsigned long long)__double_as_longlong(a));
}

// y += e (FP64 accumulation of the correction).
template <typename T>
__global__ void k_add_correction(int64_t m, double* __restrict__ yv, const T* __restrict__ e) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) yv[i] += (double)e[i];
}

// Field update (supporting information Sec. 1):
// phi^{k+1} = 2 phi^k - phi^{k-1} - (4pi/h) y*, written over phi^{k-1}.
__global__ void k_update(int64_t m, const double* __restrict__ phik, double* __restrict__ phikm1,
                         const double* __restrict__ yv, double coef) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) phikm1[i] = 2.0 * phik[i] - phikm1[i] - coef * yv[i];
}

// ---------------------------------------------------------------- multigrid
// Red-black Gauss-Seidel half sweep on M e = b: points with (x+y+z)%2 == color
// get e = (sum of neighbours - b)/6.  One thread per point of the colour.
template <typename T>
__global__ void __launch_bounds__(P3_THREADS)
k_rbgs(int n, T* __restrict__ e, const T* __restrict__ b, int color) {
    const int half = n >> 1;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)half * n * n) return;
    const int xi = (int)(t % half);
    const int64_t rr = t / half;
    const int y = (int)(rr % n), z = (int)(rr / n);
    const int x = 2 * xi + ((y + z + color) & 1);
    const int64_t i = ((int64_t)z * n + y) * n + x;
    e[i] = (nb6(e, x, y, z, n) - b[i]) * (T)(1.0 / 6.0);
}

// r = b - M e on one level.
template <typename T>
__global__ void __launch_bounds__(P3_THREADS)
k_resid(int n, const T* __restrict__ e, const T* __restrict__ b, T* __restrict__ r) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * n * n) return;
    int x, y, z;
    unflatten(i, n, x, y, z);
    r[i] = b[i] - (nb6(e, x, y, z, n) - (T)6 * e[i]);
}

// Full-weighting restriction to the coarse level (nc = n_fine/2) and the
// rediscretisation factor 4 (the coarse spacing is twice the fine one):
// b_c[I] = 4 sum_{d in {-1,0,1}^3} w(d) r_f[2I + d], w = prod (1/2 or 1/4).
template <typename T>
__global__ void __launch_bounds__(P3_THREADS)
k_restrict(int nc, const T* __restrict__ rf, T* __restrict__ bc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nc * nc * nc) return;
    int X, Y, Z;
    unflatten(i, nc, X, Y, Z);
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
            const T* row = rf + ((int64_t)z * n + y) * n;
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) acc += wyz * w1[dx + 1] * row[wrap_idx(2 * X + dx, n)];
        }
    }
    bc[i] = (T)4 * acc;
}

// Trilinear prolongation and correction on the fine level: e_f += P e_c.
template <typename T>
__global__ void __launch_bounds__(P3_THREADS)
k_prolong_add(int n, const T* __restrict__ ec, T* __restrict__ ef) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * n * n) return;
    int x, y, z;
    unflatten(i, n, x, y, z);
    const int nc = n >> 1;
    int ix[2], iy[2], iz[2];
    T wx[2], wy[2], wz[2];
    ix[0] = x >> 1; ix[1] = (x & 1) ? ((x >> 1) + 1 == nc ? 0 : (x >> 1) + 1) : ix[0];
    wx[0] = (x & 1) ? (T)0.5 : (T)1; wx[1] = (x & 1) ? (T)0.5 : (T)0;
    iy[0] = y >> 1; iy[1] = (y & 1) ? ((y >> 1) + 1 == nc ? 0 : (y >> 1) + 1) : iy[0];
    wy[0] = (y & 1) ? (T)0.5 : (T)1; wy[1] = (y & 1) ? (T)0.5 : (T)0;
    iz[0] = z >> 1; iz[1] = (z & 1) ? ((z >> 1) + 1 == nc ? 0 : (z >> 1) + 1) : iz[0];
    wz[0] = (z & 1) ? (T)0.5 : (T)1; wz[1] = (z & 1) ? (T)0.5 : (T)0;
    T acc = 0;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a)
                acc += wx[a] * wy[b] * wz[c] * ec[((int64_t)iz[c] * nc + iy[b]) * nc + ix[a]];
    ef[i] += acc;
}

// Coarsest level: e = M^+ b in FP64 with the translation-invariant
// pseudo-inverse kernel g (e_i = sum_j g[(i - j) mod n] b_j).  One block.
template <typename T>
__global__ void k_coarse_solve(int n, const double* __restrict__ g, const T* __restrict__ b, T* __restrict__ e) {
    __shared__ double sb[512];
    const int m = n * n * n;
    for (int j = threadIdx.x; j < m; j += blockDim.x) sb[j] = (double)b[j];
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int x = i % n, y = (i / n) % n, z = i / (n * n);
        double acc = 0.0;
        for (int j = 0; j < m; ++j) {
            const int jx = j % n, jy = (j / n) % n, jz = j / (n * n);
            int dx = x - jx, dy = y - jy, dz = z - jz;
            dx += dx < 0 ? n : 0;
            dy += dy < 0 ? n : 0;
            dz += dz < 0 ? n : 0;
            acc += g[(dz * n + dy) * n + dx] * sb[j];
        }
        e[i] = (T)acc;
    }
}

// ---------------------------------------------------------------- interpolation
// F_a = -ke Q_a sum_n W(r_a - r_n) (D phi)_n with central differences
// (Eq. 21), one thread per particle in cell order; writes the total force
// (adding the short-range part) and the two parts in original order.
__global__ void __launch_bounds__(P3_THREADS)
k_gather(int np, const PQ* __restrict__ xq, const int* __restrict__ order, int n, double inv_h,
         double ke, const double* __restrict__ phi, const double* __restrict__ Fsr_s,
         double* __restrict__ F, double* __restrict__ Flr, double* __restrict__ Fsr) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= np) return;
    const PQ p = xq[s];
    double wx[4], wy[4], wz[4];
    const int bx = bspline_axis(p.x, inv_h, n, wx);
    const int by = bspline_axis(p.y, inv_h, n, wy);
    const int bz = bspline_axis(p.z, inv_h, n, wz);
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int c = 0; c < 4; ++c) {
        const int iz = wrap_idx(bz + c, n);
        const int izm = iz == 0 ? n - 1 : iz - 1, izp = iz == n - 1 ? 0 : iz + 1;
        for (int b = 0; b < 4; ++b) {
            const int iy = wrap_idx(by + b, n);
            const int iym = iy == 0 ? n - 1 : iy - 1, iyp = iy == n - 1 ? 0 : iy + 1;
            const double wyz = wy[b] * wz[c];
            for (int a = 0; a < 4; ++a) {
                const int ix = wrap_idx(bx + a, n);
                const int ixm = ix == 0 ? n - 1 : ix - 1, ixp = ix == n - 1 ? 0 : ix + 1;
                const double w = wyz * wx[a];
                const int64_t row = ((int64_t)iz * n + iy) * n;
                gx += w * (phi[row + ixp] - phi[row + ixm]);
                gy += w * (phi[((int64_t)iz * n + iyp) * n + ix] - phi[((int64_t)iz * n + iym) * n + ix]);
                gz += w * (phi[((int64_t)izp * n + iy) * n + ix] - phi[((int64_t)izm * n + iy) * n + ix]);
            }
        }
    }
    const double scale = -ke * p.w * 0.5 * inv_h;
    const int i = order[s];
    const double f[3] = {scale * gx, scale * gy, scale * gz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double sr = Fsr_s[3 * s + d];
        F[3 * i + d] = sr + f[d];
        Flr[3 * i + d] = f[d];
        Fsr[3 * i + d] = sr;
    }
}

}  // namespace p3
