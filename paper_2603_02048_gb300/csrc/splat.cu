// Particle -> grid density splat (Sec. 3.3.1 of arXiv 2603.02048):
// rho(x_v) = sum_p m_p W(|x_v - x_p|, h) at voxel centres, W the M4 cubic
// spline with support 2h.
//
// One warp per particle. Each lane owns an (x, y) column of the particle's
// footprint (the voxels whose centres lie within 2h on every axis: 8^3 for
// h = 2), the lanes forming an 8 (x) by 4 (y) grid, and walks the column in
// z with the column's squared distance computed once; at every z slice a
// warp's atomics cover four 8-float rows (four 32-byte sectors) and compile
// to fire-and-forget reductions in L2. Columns and voxels beyond the support
// (r^2 >= 4h^2, about half of the footprint box) skip the square root and the
// atomic; indices are 32-bit (grids hold fewer than 2^31 voxels).
#include "hh_internal.h"

namespace hh {
namespace {

// M4 cubic spline, q = r / h: norm (1 - 3/2 q^2 + 3/4 q^3) on [0,1),
// norm (2 - q)^3 / 4 on [1,2), 0 beyond; norm = 1 / (pi h^3). Both pieces are
// evaluated and selected, so lanes on either side of q = 1 do not diverge.
__device__ __forceinline__ float m4_kernel(float r, float inv_h, float norm) {
    const float q = r * inv_h;
    const float inner = fmaf(q * q, fmaf(0.75f, q, -1.5f), 1.0f);
    const float t = fmaxf(2.0f - q, 0.0f);
    const float outer = 0.25f * t * t * t;
    return norm * (q < 1.0f ? inner : outer);
}

// Hardware approximate square root (PTX sqrt.approx.f32, ~1 ulp).
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
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
    if (x1 < x0 || y1 < y0 || z1 < z0) return;
    const int lx = lane & 7, ly = lane >> 3;
    const float reach2 = 4.0f * h * h;
    const float m = q.w;
    const int ez = z1 - z0 + 1;
    const unsigned plane = static_cast<unsigned>(nx) * static_cast<unsigned>(ny);
    const float dz0 = (static_cast<float>(z0) + 0.5f) - q.z;
    for (int yb = y0; yb <= y1; yb += 4) {
        for (int xb = x0; xb <= x1; xb += 8) {
            const int i = xb + lx, j = yb + ly;
            if (i > x1 || j > y1) continue;
            const float dx = (static_cast<float>(i) + 0.5f) - q.x;
            const float dy = (static_cast<float>(j) + 0.5f) - q.y;
            const float dxy2 = fmaf(dx, dx, dy * dy);
            if (!(dxy2 < reach2)) continue;  // the whole column is outside the support
            float* col = rho + (static_cast<unsigned>(z0) * static_cast<unsigned>(ny) +
                                static_cast<unsigned>(j)) * static_cast<unsigned>(nx) + i;
            float dz = dz0;  // (k + 1/2) - z exactly: each +1 is exact at these magnitudes
            for (int k = 0; k < ez; ++k, dz += 1.0f, col += plane) {
                const float r2 = fmaf(dz, dz, dxy2);
                if (r2 < reach2) {
                    const float w = m4_kernel(sqrt_approx(r2), inv_h, norm);
                    if (w > 0.0f) atomicAdd(col, m * w);
                }
            }
        }
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
