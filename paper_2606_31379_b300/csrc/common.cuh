// Shared device helpers and constants of the P3MaZe CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define P3_THREADS 256

// Unit conversion: (kcal/mol/A) / (g/mol) -> A/fs^2.
#define P3_ACCEL 4.184e-4
// Default Coulomb constant, kcal A / (mol e^2).
#define P3_COULOMB_K 332.0637

namespace p3 {

// Cell-ordered particle record (x, y, z, Q): one 32-byte aligned load.
struct __align__(32) PQ {
    double x, y, z, w;
};

constexpr double kPi = 3.14159265358979323846;
constexpr double kTwoOverSqrtPi = 1.12837916709551257390;

// Periodic wrap of an index known to lie in [-n, 2n).
__device__ __forceinline__ int wrap_idx(int i, int n) {
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

// Cubic (order-4) B-spline weights of the nodes floor(u)-1 .. floor(u)+2 for a
// fractional offset t = u - floor(u) (charge assignment, Sec. 2).
__device__ __forceinline__ void bspline4(double t, double w[4]) {
    const double s = 1.0 - t;
    const double t2 = t * t, t3 = t2 * t;
    w[0] = s * s * s * (1.0 / 6.0);
    w[1] = (3.0 * t3 - 6.0 * t2 + 4.0) * (1.0 / 6.0);
    w[2] = (-3.0 * t3 + 3.0 * t2 + 3.0 * t + 1.0) * (1.0 / 6.0);
    w[3] = t3 * (1.0 / 6.0);
}

// Base node (floor(u) - 1, wrapped into [0, n)) and weights along one axis.
__device__ __forceinline__ int bspline_axis(double x, double inv_h, int n, double w[4]) {
    double u = x * inv_h;
    // positions are wrapped into [0, L); a non-finite one maps to node 0 so
    // every access stays in bounds (the NaN charge weight then surfaces as a
    // non-finite constraint residual)
    if (!(u >= 0.0 && u <= (double)n)) u = 0.0;
    const double f = floor(u);
    bspline4(u - f, w);
    int b = (int)f - 1;
    return b < 0 ? b + n : (b >= n ? b - n : b);
}

// FP32 weights of the cubic B-spline at fraction t in [0, 1) (the same
// polynomials as bspline4).
__device__ __forceinline__ void bspline4f(float t, float w[4]) {
    const float s = 1.0f - t;
    const float t2 = t * t, t3 = t2 * t;
    w[0] = s * s * s * (1.0f / 6.0f);
    w[1] = (3.0f * t3 - 6.0f * t2 + 4.0f) * (1.0f / 6.0f);
    w[2] = (-3.0f * t3 + 3.0f * t2 + 3.0f * t + 1.0f) * (1.0f / 6.0f);
    w[3] = t3 * (1.0f / 6.0f);
}

// d/dt of the four weights (derivatives of the polynomials above; they sum
// to zero), FP64 and FP32.
__device__ __forceinline__ void bspline4_deriv(double t, double d[4]) {
    const double s = 1.0 - t;
    d[0] = -0.5 * s * s;
    d[1] = (1.5 * t - 2.0) * t;
    d[2] = (-1.5 * t + 1.0) * t + 0.5;
    d[3] = 0.5 * t * t;
}
__device__ __forceinline__ void bspline4f_deriv(float t, float d[4]) {
    const float s = 1.0f - t;
    d[0] = -0.5f * s * s;
    d[1] = (1.5f * t - 2.0f) * t;
    d[2] = (-1.5f * t + 1.0f) * t + 0.5f;
    d[3] = 0.5f * t * t;
}

// A particle's mesh coordinates for FP32 assignment and interpolation: base
// node per axis (as bspline_axis), the fractions u - floor(u) rounded once
// to FP32 (the FP64 part is done once per particle and step), and Q.
struct __align__(32) MeshPt {
    int bx, by, bz;
    float q;
    float tx, ty, tz;
    float pad;
};

__device__ __forceinline__ int mesh_axis(double x, double inv_h, int n, float* t) {
    double u = x * inv_h;
    if (!(u >= 0.0 && u <= (double)n)) u = 0.0;
    const double f = floor(u);
    *t = (float)(u - f);
    const int b = (int)f - 1;
    return b < 0 ? b + n : (b >= n ? b - n : b);
}

// Programmatic dependent launch (sm_90+): a kernel launched with the
// programmatic-serialization attribute may be scheduled before its
// predecessor in the stream has finished.  pdl_wait() blocks until the
// predecessor grid has completed and its memory is visible; pdl_trigger()
// lets the successor grid be scheduled (its blocks then wait in their own
// pdl_wait()).  Both are no-ops for a kernel launched without the attribute.
// Every kernel that the library launches with the attribute calls pdl_wait()
// before its first access to memory that a predecessor reads or writes
// (reads of constant tables may come first), then pdl_trigger(); the
// trigger only lets the successor's blocks be scheduled, its wait still
// holds them until this grid has completed.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ int linear_tid() {
    return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}

__device__ __forceinline__ int block_threads() { return blockDim.x * blockDim.y * blockDim.z; }

// Block-wide sum of a double (all threads get the result).  Any block shape.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int tid = linear_tid(), lane = tid & 31, wid = tid >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (block_threads() + 31) >> 5;
    v = (tid < nw) ? sh[tid] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (tid == 0) sh[0] = v;
    __syncthreads();
    v = sh[0];
    __syncthreads();
    return v;
}

__device__ __forceinline__ double block_max(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int tid = linear_tid(), lane = tid & 31, wid = tid >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    const int nw = (block_threads() + 31) >> 5;
    v = (tid < nw) ? sh[tid] : 0.0;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (tid == 0) sh[0] = v;
    __syncthreads();
    v = sh[0];
    __syncthreads();
    return v;
}

// Block-wide maximum of a float (all threads get the result).  Any block shape.
__device__ __forceinline__ float block_max_f(float v) {
    __shared__ float shf[32];
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int tid = linear_tid(), lane = tid & 31, wid = tid >> 5;
    __syncthreads();
    if (lane == 0) shf[wid] = v;
    __syncthreads();
    const int nw = (block_threads() + 31) >> 5;
    v = (tid < nw) ? shf[tid] : 0.0f;
    if (wid == 0)
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (tid == 0) shf[0] = v;
    __syncthreads();
    v = shf[0];
    __syncthreads();
    return v;
}

}  // namespace p3
