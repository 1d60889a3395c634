// Particle -> grid density splat (Sec. 3.3.1 of arXiv 2603.02048):
// rho(x_v) = sum_p m_p W(|x_v - x_p|, h) at voxel centres, W the M4 cubic
// spline with support 2h.
//
// Two kernels: splat_box8_kernel for supports of at most 8 voxels per axis
// (2h <= 4, the paper's h = 2), described where it is defined, and
// splat_warp_kernel for wider ones. Both put four particles on a warp,
// eight lanes each, so that a warp's reductions at one (y, z) row cover four
// 8-float runs (four 32-byte sectors, one per particle) and compile to
// fire-and-forget reductions in L2, and the per-particle set-up is shared by
// the four particles' lanes (against one particle per warp this took 12 %
// off the build; eight per warp, half-sector reductions, was slower again).
//
// splat_warp_kernel: a lane owns an (x, y) column of its particle's
// footprint (the voxels whose centres lie within 2h on every axis), the
// eight lanes covering a row of 8 columns per pass, and walks the column in z
// with the column's squared distance computed once. Columns and voxels
// beyond the support (r^2 >= 4h^2) skip the atomic; indices are 32-bit
// (grids hold fewer than 2^31 voxels). The kernel is evaluated in r with the
// particle's mass folded into its coefficients.
#include <algorithm>

#include "hh_internal.h"

namespace hh {
namespace {

// m W(r, h) for the M4 cubic spline with the particle mass folded in:
// W = norm (1 - 3/2 q^2 + 3/4 q^3) on q = r/h < 1, norm (2 - q)^3 / 4 on
// [1, 2), norm = 1 / (pi h^3); in r: m W = mn + r^2 (c2 + c3 r) for r < h and
// d (2h - r)^3 beyond, mn = m norm, c2 = -3/2 mn / h^2, c3 = 3/4 mn / h^3,
// d = mn / (4 h^3). Both pieces are evaluated and selected (no divergence).
struct M4Coef {
    float mn, c2, c3, d, h, two_h;
};

__device__ __forceinline__ M4Coef m4_coef(float m, float h, float inv_h, float norm) {
    M4Coef c;
    c.mn = m * norm;
    const float inv_h2 = inv_h * inv_h, inv_h3 = inv_h2 * inv_h;
    c.c2 = -1.5f * c.mn * inv_h2;
    c.c3 = 0.75f * c.mn * inv_h3;
    c.d = 0.25f * c.mn * inv_h3;
    c.h = h;
    c.two_h = 2.0f * h;
    return c;
}

__device__ __forceinline__ float m4_mass(const M4Coef& c, float r2, float r) {
    const float inner = fmaf(r2, fmaf(c.c3, r, c.c2), c.mn);
    const float t = fmaxf(c.two_h - r, 0.0f);
    const float outer = c.d * (t * t * t);
    return r < c.h ? inner : outer;
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

constexpr int kParticlesPerWarp = 4;

template <int PPW>  // particles per warp: 32 / PPW lanes each
__global__ void __launch_bounds__(256) splat_warp_kernel(const float4* __restrict__ parts,
                                                         int64_t n, int nx, int ny, int nz,
                                                         float h, float inv_h, float norm,
                                                         float* __restrict__ rho) {
    constexpr int LPP = 32 / PPW;               // lanes per particle
    constexpr int COLS = LPP >= 8 ? 8 : LPP;    // footprint columns per pass along x
    constexpr int ROWS = LPP / COLS;            // footprint rows per pass
    const int lane = threadIdx.x & 31;
    const int64_t p =
        ((static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * PPW + lane / LPP;
    if (p >= n) return;
    const float4 q = __ldg(parts + p);
    int x0, x1, y0, y1, z0, z1;
    footprint(q.x, 2.0f * h, nx, x0, x1);
    footprint(q.y, 2.0f * h, ny, y0, y1);
    footprint(q.z, 2.0f * h, nz, z0, z1);
    if (x1 < x0 || y1 < y0 || z1 < z0) return;
    const int sl = lane % LPP;
    const int lx = sl % COLS, ly = sl / COLS;
    const float reach2 = 4.0f * h * h;
    const M4Coef cf = m4_coef(q.w, h, inv_h, norm);
    const int ez = z1 - z0 + 1;
    const unsigned plane = static_cast<unsigned>(nx) * static_cast<unsigned>(ny);
    const float dz0 = (static_cast<float>(z0) + 0.5f) - q.z;
    for (int yb = y0; yb <= y1; yb += ROWS) {
        for (int xb = x0; xb <= x1; xb += COLS) {
            const int i = xb + lx, j = yb + ly;
            if (i > x1 || j > y1) continue;
            const float dx = (static_cast<float>(i) + 0.5f) - q.x;
            const float dy = (static_cast<float>(j) + 0.5f) - q.y;
            const float dxy2 = fmaf(dx, dx, dy * dy);
            if (!(dxy2 < reach2)) continue;  // the whole column is outside the support
            unsigned v = (static_cast<unsigned>(z0) * static_cast<unsigned>(ny) +
                          static_cast<unsigned>(j)) * static_cast<unsigned>(nx) + i;
            float dz = dz0;  // (k + 1/2) - z exactly: each +1 is exact at these magnitudes
            for (int k = 0; k < ez; ++k, dz += 1.0f, v += plane) {
                const float r2 = fmaf(dz, dz, dxy2);
                if (r2 < reach2) atomicAdd(rho + v, m4_mass(cf, r2, sqrt_approx(r2)));
            }
        }
    }
}

// Adds v to the float at byte address addr when t > 0 (a predicated
// reduction: no branch, nothing issued to memory otherwise).
__device__ __forceinline__ void red_add_if_positive(float t, uint64_t addr, float v) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.gt.f32 p, %0, 0f00000000;\n\t"
                 "@p red.global.add.f32 [%1], %2;\n\t}"
                 :: "f"(t), "l"(addr), "f"(v) : "memory");
}

// PTX sqrt.approx.ftz.f32: a subnormal r^2 is taken as 0 (r ~ 0 there,
// where W is flat), which keeps the instruction free of a subnormal path.
__device__ __forceinline__ float sqrt_approx_ftz(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// a * b + c with a 32 x 32 -> 64-bit product (PTX mad.wide.u32).
__device__ __forceinline__ uint64_t mad_wide(uint32_t a, uint32_t b, uint64_t c) {
    uint64_t r;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(a), "r"(b), "l"(c));
    return r;
}

// First of the 8 voxel slots along one axis that cover every voxel centre
// within `reach` (<= 4) of x: the smallest k with k + 1/2 > x - reach,
// clamped to [-8, n] so that the slots' indices stay small (slots outside
// [0, n) are masked by their distance; NaN converts to 0 and is masked the
// same way).
__device__ __forceinline__ int box8_start(float x, float reach, int n) {
    const float a = fminf(fmaxf(x - reach - 0.5f, -9.0f), static_cast<float>(n));
    return __float2int_rd(a) + 1;
}

// Distance from x to the centre of voxel k, infinite when k lies outside
// [0, n).
__device__ __forceinline__ float dist_or_inf(int k, int n, float x) {
    return (k >= 0 && k < n) ? (static_cast<float>(k) + 0.5f) - x : __int_as_float(0x7f800000);
}

// The splat for kernel radii 2h <= 4 voxels (the paper's h = 2 among them):
// every particle's support fits an 8 x 8 x 8 box of voxel slots. Four
// particles per warp, eight lanes each on the box's x slots; a lane walks its
// 8 y rows and 8 z slots fully unrolled. Slots outside the grid get an
// infinite distance, so no index test is needed per slot, and a slot adds
// its mass only where it lies inside the support (a predicated reduction, no
// branch). The kernel is evaluated in the branch-free form
// m W = m norm (2 t^3 - u^3), t = 1 - r/2h, u = max(1 - r/h, 0), equal to the
// two-piece M4 on [0, 2h): 2 t^3 = (2 - q)^3 / 4 and u^3 = (1 - q)^3 for
// q = r/h < 1. Against splat_warp_kernel (per-column and per-voxel branches,
// the footprint walked in loops) this issues a third fewer instructions and
// the 256^3 plume's splat drops from 120 to 91 us; packed FP32x2 arithmetic
// for slot pairs issues fewer still but is no faster, the L2 reductions now
// setting the pace.
template <int PPW>
__global__ void __launch_bounds__(256) splat_box8_kernel(const float4* __restrict__ parts,
                                                         int64_t n, int nx, int ny, int nz,
                                                         float reach, float inv_2h, float inv_h,
                                                         float norm, float* __restrict__ rho) {
    constexpr int LPP = 32 / PPW;
    static_assert(LPP == 8, "eight lanes per particle: one per x slot");
    const int lane = threadIdx.x & 31;
    const int64_t p =
        ((static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * PPW + lane / LPP;
    if (p >= n) return;
    const float4 q = __ldg(parts + p);
    const int sx = box8_start(q.x, reach, nx), sy = box8_start(q.y, reach, ny),
              sz = box8_start(q.z, reach, nz);
    const int i = sx + (lane % LPP);
    const float dx = dist_or_inf(i, nx, q.x);
    const float dx2 = dx * dx;
    float dz[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) dz[k] = dist_or_inf(sz + k, nz, q.z);
    const float mn = q.w * norm, c_t = 2.0f * mn, c_u = -mn;
    const uint64_t row_b = static_cast<uint64_t>(nx) * sizeof(float);
    // a plane is at most 16384^2 floats (1 GiB): its byte size fits 32 bits
    const uint32_t plane_b = static_cast<uint32_t>(row_b * static_cast<uint64_t>(ny));
    // byte address of slot (i, sy, sz); unsigned arithmetic, formed for
    // masked slots too but never dereferenced there
    uint64_t row = reinterpret_cast<uint64_t>(rho) +
                   static_cast<uint64_t>((static_cast<int64_t>(sz) * ny + sy) * nx + i) *
                       sizeof(float);
#pragma unroll
    for (int j = 0; j < 8; ++j, row += row_b) {
        const float dy = dist_or_inf(sy + j, ny, q.y);
        const float dxy2 = fmaf(dy, dy, dx2);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float r = sqrt_approx_ftz(fmaf(dz[k], dz[k], dxy2));
            const float t = fmaf(r, -inv_2h, 1.0f);
            const float u = __saturatef(fmaf(r, -inv_h, 1.0f));
            const float w = fmaf(t * t * t, c_t, (u * u * u) * c_u);
            red_add_if_positive(t, mad_wide(plane_b, k, row), w);
        }
    }
}

// Binning for the splat of grids larger than L2. Particles arrive in any
// order; splatted in that order, concurrent warps scatter their reductions
// over the whole density grid, and once the grid outgrows L2 most of them
// miss it. Sorted by cell (a counting sort: count, one-block exclusive scan,
// scatter with per-bin cursors), the warps in flight cover a few cells and
// the reductions stay in L2. A cell is at least 16 voxels wide and at most
// 64 cells span an axis (at most 2^18 cells).
struct BinGeom {
    int nbx, nby, nbz;
    float inv;  // 1 / cell width
};

__host__ __device__ inline BinGeom bin_geom(int nx, int ny, int nz) {
    const int m = nx > ny ? (nx > nz ? nx : nz) : (ny > nz ? ny : nz);
    int w = (m + 63) / 64;
    if (w < 16) w = 16;
    BinGeom g;
    g.nbx = (nx + w - 1) / w;
    g.nby = (ny + w - 1) / w;
    g.nbz = (nz + w - 1) / w;
    g.inv = 1.0f / static_cast<float>(w);
    return g;
}

// Cell of a particle; positions outside the grid (and NaN, which converts to
// 0) go to the nearest edge cell: the order is all that matters.
__device__ __forceinline__ int bin_of(const float4& p, const BinGeom& g) {
    const int bx = min(max(__float2int_rd(p.x * g.inv), 0), g.nbx - 1);
    const int by = min(max(__float2int_rd(p.y * g.inv), 0), g.nby - 1);
    const int bz = min(max(__float2int_rd(p.z * g.inv), 0), g.nbz - 1);
    return (bz * g.nby + by) * g.nbx + bx;
}

__global__ void bin_count_kernel(const float4* __restrict__ parts, int64_t n, BinGeom g,
                                 unsigned* __restrict__ count) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        atomicAdd(count + bin_of(__ldg(parts + i), g), 1u);
}

// Exclusive prefix sum of count[0..nb) into offset[0..nb), one block of 1024
// threads, each owning a contiguous chunk (a multiple of 4 counters). When
// nb is a multiple of 4 and a chunk at most 32, a thread holds its chunk in
// registers, loaded and stored as 16-byte vectors; otherwise it walks it.
__global__ void __launch_bounds__(1024) bin_scan_kernel(const unsigned* __restrict__ count,
                                                        unsigned* __restrict__ offset, int nb) {
    __shared__ unsigned warp_sum[32];
    constexpr int kVec = 8;  // 16-byte vectors a thread holds
    const int t = threadIdx.x;
    const int chunk = (((nb + 1023) / 1024) + 3) & ~3;
    const bool vec = (nb & 3) == 0 && chunk <= 4 * kVec;
    const int b0 = min(t * chunk, nb), b1 = min(b0 + chunk, nb);
    uint4 v[kVec];
    unsigned sum = 0;
    if (vec) {
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
            v[j] = b0 + 4 * j < b1 ? reinterpret_cast<const uint4*>(count + b0)[j]
                                   : make_uint4(0u, 0u, 0u, 0u);
            sum += v[j].x + v[j].y + v[j].z + v[j].w;
        }
    } else {
        for (int b = b0; b < b1; ++b) sum += count[b];
    }
    // inclusive scan of the per-thread sums across the block
    unsigned x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if ((t & 31) >= o) x += y;
    }
    if ((t & 31) == 31) warp_sum[t >> 5] = x;
    __syncthreads();
    if (t < 32) {
        unsigned w = warp_sum[t];
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
            if (t >= o) w += y;
        }
        warp_sum[t] = w;
    }
    __syncthreads();
    unsigned run = x - sum + ((t >> 5) ? warp_sum[(t >> 5) - 1] : 0u);  // exclusive
    if (vec) {
#pragma unroll
        for (int j = 0; j < kVec; ++j) {
            if (b0 + 4 * j < b1) {
                uint4 o;
                o.x = run;
                o.y = o.x + v[j].x;
                o.z = o.y + v[j].y;
                o.w = o.z + v[j].z;
                run = o.w + v[j].w;
                reinterpret_cast<uint4*>(offset + b0)[j] = o;
            }
        }
    } else {
        for (int b = b0; b < b1; ++b) {
            offset[b] = run;
            run += count[b];
        }
    }
}

__global__ void bin_scatter_kernel(const float4* __restrict__ parts, int64_t n, BinGeom g,
                                   unsigned* __restrict__ cursor, float4* __restrict__ sorted) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float4 p = __ldg(parts + i);
        sorted[atomicAdd(cursor + bin_of(p, g), 1u)] = p;
    }
}

}  // namespace

int splat_bin_count(int nx, int ny, int nz) {
    const BinGeom g = bin_geom(nx, ny, nz);
    return g.nbx * g.nby * g.nbz;
}

cudaError_t launch_bin_particles(const float4* xyzm, int64_t n, int nx, int ny, int nz,
                                 unsigned* bins, float4* sorted, cudaStream_t s) {
    const BinGeom g = bin_geom(nx, ny, nz);
    const int nb = g.nbx * g.nby * g.nbz;
    cudaError_t e = cudaMemsetAsync(bins, 0, static_cast<size_t>(nb) * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const int threads = 256;
    // grid-stride kernels: at most 16 resident 256-thread blocks per SM
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 1;
    const unsigned blocks = static_cast<unsigned>(std::min<int64_t>((n + threads - 1) / threads,
                                                                    int64_t(sms) * 16));
    bin_count_kernel<<<blocks, threads, 0, s>>>(xyzm, n, g, bins);
    bin_scan_kernel<<<1, 1024, 0, s>>>(bins, bins + nb, nb);
    bin_scatter_kernel<<<blocks, threads, 0, s>>>(xyzm, n, g, bins + nb, sorted);
    count_launch(3);
    return cudaGetLastError();
}

cudaError_t launch_splat(const float4* xyzm, int64_t n, int nx, int ny, int nz, float h,
                         float* rho, cudaStream_t s) {
    const size_t nvox = static_cast<size_t>(nx) * ny * nz;
    cudaError_t e = cudaMemsetAsync(rho, 0, nvox * sizeof(float), s);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t warps = (n + kParticlesPerWarp - 1) / kParticlesPerWarp;
    const int64_t blocks = (warps * 32 + threads - 1) / threads;
    const double hd = h;
    const float norm = static_cast<float>(1.0 / (3.14159265358979323846 * hd * hd * hd));
    if (2.0 * hd <= 4.0)
        splat_box8_kernel<kParticlesPerWarp><<<static_cast<unsigned>(blocks), threads, 0, s>>>(
            xyzm, n, nx, ny, nz, 2.0f * h, static_cast<float>(0.5 / hd),
            static_cast<float>(1.0 / hd), norm, rho);
    else
        splat_warp_kernel<kParticlesPerWarp><<<static_cast<unsigned>(blocks), threads, 0, s>>>(
            xyzm, n, nx, ny, nz, h, static_cast<float>(1.0 / hd), norm, rho);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hh
