// Particle -> grid density splat (Sec. 3.3.1 of arXiv 2603.02048):
// rho(x_v) = sum_p m_p W(|x_v - x_p|, h) at voxel centres, W the M4 cubic
// spline with support 2h.
//
// One warp per particle. The lanes walk the particle's footprint (the voxels
// whose centres lie within 2h on every axis: 8^3 for h = 2) x-fastest, so a
// warp's 32 atomics cover four 8-float rows (four 32-byte sectors) and
// compile to fire-and-forget reductions in L2.
#include "hh_internal.h"

namespace hh {
namespace {

// M4 cubic spline, q = r / h: norm (1 - 3/2 q^2 + 3/4 q^3) on [0,1),
// norm (2 - q)^3 / 4 on [1,2), 0 beyond; norm = 1 / (pi h^3).
__device__ __forceinline__ float m4_kernel(float r, float inv_h, float norm) {
    float q = r * inv_h;
    if (q < 1.0f) return norm * (1.0f - 1.5f * q * q + 0.75f * q * q * q);
    if (q < 2.0f) {
        float t = 2.0f - q;
        return norm * 0.25f * t * t * t;
    }
    return 0.0f;
}

// First and last voxel index along one axis whose centre lies within `reach`
// of x, clipped to [0, n-1] (empty when lo > hi; NaN gives an empty range).
__device__ __forceinline__ void footprint(float x, float reach, int n, int& lo, int& hi) {
    float a = fminf(fmaxf(x - reach - 0.5f, -1.0f), (float)n);
    float b = fminf(fmaxf(x + reach - 0.5f, -1.0f), (float)n);
    lo = max(0, (int)ceilf(a));
    hi = min(n - 1, (int)floorf(b));
}

__global__ void __launch_bounds__(256) splat_warp_kernel(const float4* __restrict__ parts,
                                                         int64_t n, int nx, int ny, int nz,
                                                         float h, float inv_h, float norm,
                                                         float* __restrict__ rho) {
    const int64_t p = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= n) return;
    const float4 q = __ldg(parts + p);
    int x0, x1, y0, y1, z0, z1;
    footprint(q.x, 2.0f * h, nx, x0, x1);
    footprint(q.y, 2.0f * h, ny, y0, y1);
    footprint(q.z, 2.0f * h, nz, z0, z1);
    const int ex = x1 - x0 + 1, ey = y1 - y0 + 1, ez = z1 - z0 + 1;
    if (ex <= 0 || ey <= 0 || ez <= 0) return;
    const int plane = ex * ey;
    const int total = plane * ez;
    for (int t = lane; t < total; t += 32) {
        const int k = t / plane;
        const int r = t - k * plane;
        const int j = r / ex;
        const int i = r - j * ex;
        const int gi = x0 + i, gj = y0 + j, gk = z0 + k;
        const float dx = (static_cast<float>(gi) + 0.5f) - q.x;
        const float dy = (static_cast<float>(gj) + 0.5f) - q.y;
        const float dz = (static_cast<float>(gk) + 0.5f) - q.z;
        const float w = m4_kernel(sqrtf(dx * dx + dy * dy + dz * dz), inv_h, norm);
        if (w > 0.0f)
            atomicAdd(rho + (static_cast<size_t>(gk) * ny + gj) * nx + gi, q.w * w);
    }
}

}  // namespace

cudaError_t launch_splat(const float4* xyzm, int64_t n, int nx, int ny, int nz, float h,
                         float* rho, cudaStream_t s) {
    const size_t nvox = static_cast<size_t>(nx) * ny * nz;
    cudaError_t e = cudaMemsetAsync(rho, 0, nvox * sizeof(float), s);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (n * 32 + threads - 1) / threads;
    const double hd = h;
    const float norm = static_cast<float>(1.0 / (3.14159265358979323846 * hd * hd * hd));
    splat_warp_kernel<<<static_cast<unsigned>(blocks), threads, 0, s>>>(
        xyzm, n, nx, ny, nz, h, static_cast<float>(1.0 / hd), norm, rho);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hh
