// Diffusion smoothing of a caller-owned mesh that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// smoothing: code that runs under a fixed device-memory budget handed out by
// a host framework that owns every allocation (a cudaMalloc behind its back
// would break its accounting, or fail once the budget is taken), and
// long-running services that reserve their device memory at start-up and
// must not grow the process's footprint afterwards.  This entry point serves
// them: the caller passes the input and output meshes, and the only scratch
// (a ping-pong mesh and the block partial sums of the neutrality mean) lives
// in one file-scope device array below, reserved on every GPU that loads this
// library until the process exits.
#include "p3maze.h"

#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "mesh.cuh"

using namespace p3;

// Defined in p3maze.cu: the message returned by p3maze_last_error(NULL).
void p3_set_global_error(const char* msg);

namespace {

constexpr int kNoAllocMaxMesh = 64;                                   // points per axis
constexpr int kNoAllocMesh = kNoAllocMaxMesh * kNoAllocMaxMesh * kNoAllocMaxMesh;
constexpr int kNoAllocPartials = 4096;                                // >= blocks of one diffusion launch at 64^3 (16 at zc 8)
constexpr int kMaxDevices = 64;

// Scratch: one ping-pong mesh (FP64) followed by the FP64 block sums and the
// reduced total.  Every call on a device shares it.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMesh + kNoAllocPartials + 16];

std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

// [a, a + an) and [b, b + bn) share a byte.
bool overlap(const void* a, size_t an, const void* b, size_t bn) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bn && y < x + an;
}

int na_fail(int code, const char* msg) {
    p3_set_global_error(msg);  // read back with p3maze_last_error(NULL)
    return code;
}

// Subtract the mean sum/m from every point.
__global__ void k_sub_mean(int64_t m, double* __restrict__ x, const double* __restrict__ sum) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) x[i] -= sum[0] / (double)m;
}

// Device address of the scratch array for the current device.  The array's
// name in host code is only a host-side stand-in, so the address is looked up
// with cudaGetSymbolAddress once per device, with that device current, and
// kept for the life of the process (a cudaDeviceReset in between would leave
// it stale: calls must not span a reset of the device).
int scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(P3MAZE_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return na_fail(P3MAZE_ERR_INVALID, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return na_fail(P3MAZE_ERR_CUDA, cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return P3MAZE_OK;
}

}  // namespace

extern "C" int p3maze_smooth_noalloc(const double* q, double* qs, int32_t mesh, int32_t steps, double coeff,
                                     void* cuda_stream) {
    if (!q || !qs) return na_fail(P3MAZE_ERR_INVALID, "q and qs must be device pointers");
    if (mesh < 4 || mesh > kNoAllocMaxMesh)
        return na_fail(P3MAZE_ERR_INVALID, "mesh must be 4..64 points per axis (fixed scratch of 2 MiB)");
    const size_t bytes = sizeof(double) * (size_t)mesh * mesh * mesh;
    if (overlap(q, bytes, qs, bytes)) return na_fail(P3MAZE_ERR_INVALID, "q and qs must not overlap");
    if (steps < 0) return na_fail(P3MAZE_ERR_INVALID, "steps must be >= 0");
    if (!(coeff > 0.0 && coeff <= 1.0 / 6.0) && steps > 0)
        return na_fail(P3MAZE_ERR_INVALID, "coeff must lie in (0, 1/6]");
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    if (overlap(q, bytes, scratch, sizeof(g_noalloc_scratch)) || overlap(qs, bytes, scratch, sizeof(g_noalloc_scratch)))
        return na_fail(P3MAZE_ERR_INVALID, "q and qs must not overlap the library's scratch array");
    double* tmp = scratch;
    double* partial = scratch + kNoAllocMesh;
    double* total = partial + kNoAllocPartials;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int n = mesh;
    const int64_t m = (int64_t)n * n * n;
    const dim3 blk(P3_BX, P3_BY, 1);
    const int zc = 8;
    const dim3 grd((n + P3_BX - 1) / P3_BX, (n + P3_BY - 1) / P3_BY, (n + zc - 1) / zc);
    const int nb = (int)(grd.x * grd.y * grd.z);
    if (steps == 0) {
        cudaError_t e = cudaMemcpyAsync(qs, q, sizeof(double) * m, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return na_fail(P3MAZE_ERR_CUDA, cudaGetErrorString(e));
        k_sum_partial<double><<<64, P3_THREADS, 0, s>>>(m, qs, partial);
        k_sum_final<<<1, P3_THREADS, 0, s>>>(64, partial, total);
    } else {
        // ping-pong between the scratch mesh and qs so the last step lands in qs
        const double* src = q;
        for (int k = 0; k < steps; ++k) {
            double* dst = ((steps - 1 - k) % 2 == 0) ? qs : tmp;
            if (k == steps - 1)
                k_diffuse<double, true><<<grd, blk, 0, s>>>(n, zc, src, dst, coeff, partial);
            else
                k_diffuse<double, false><<<grd, blk, 0, s>>>(n, zc, src, dst, coeff, nullptr);
            src = dst;
        }
        k_sum_final<<<1, 1024, 0, s>>>(nb, partial, total);
    }
    k_sub_mean<<<(unsigned)((m + P3_THREADS - 1) / P3_THREADS), P3_THREADS, 0, s>>>(m, qs, total);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(P3MAZE_ERR_CUDA, cudaGetErrorString(e));
    return P3MAZE_OK;
}
