// Refractive-index volume from density (Sec. 3.3.1 of arXiv 2603.02048):
// Gladstone-Dale dn = n - 1 = K rho (Eq. 12) and g = grad n = K grad rho
// (Eq. 13) by finite differences: central inside, one-sided on the first and
// last voxel of each axis. Packed per voxel as {dn, gx, gy, gz}:
//   FP32: float4, 16 B/voxel (one pass: read rho, write the volume);
//   FP16: four halves, 8 B/voxel, dn / s_n and g / s_g with per-volume scales
//         s = max|.| / 16384 (pass 1 reduces the maxima, pass 2 recomputes the
//         differences and quantises; rho is read twice, nothing else stored).
// Threads map to voxels x-fastest in 32x8 tiles of one z slice, so every
// load of rho (centre and six neighbours) is coalesced and served from L1/L2.
#include "hh_internal.h"

namespace hh {
namespace {

struct Cell {
    float dn, gx, gy, gz;
};

__device__ __forceinline__ Cell index_cell(const float* __restrict__ rho, int i, int j, int k,
                                           int nx, int ny, int nz, float K) {
    const size_t sy = nx, sz = static_cast<size_t>(nx) * ny;
    const size_t v = k * sz + j * sy + i;
    Cell c;
    const float d0 = K * __ldg(rho + v);
    c.dn = d0;
    // x
    if (i == 0) c.gx = K * __ldg(rho + v + 1) - d0;
    else if (i == nx - 1) c.gx = d0 - K * __ldg(rho + v - 1);
    else c.gx = (K * __ldg(rho + v + 1) - K * __ldg(rho + v - 1)) * 0.5f;
    // y
    if (j == 0) c.gy = K * __ldg(rho + v + sy) - d0;
    else if (j == ny - 1) c.gy = d0 - K * __ldg(rho + v - sy);
    else c.gy = (K * __ldg(rho + v + sy) - K * __ldg(rho + v - sy)) * 0.5f;
    // z
    if (k == 0) c.gz = K * __ldg(rho + v + sz) - d0;
    else if (k == nz - 1) c.gz = d0 - K * __ldg(rho + v - sz);
    else c.gz = (K * __ldg(rho + v + sz) - K * __ldg(rho + v - sz)) * 0.5f;
    return c;
}

__global__ void __launch_bounds__(256) field_fp32_kernel(const float* __restrict__ rho, int nx,
                                                         int ny, int nz, float K,
                                                         float4* __restrict__ out,
                                                         float* __restrict__ scales) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x < 2 &&
        threadIdx.y == 0)
        scales[threadIdx.x] = 1.0f;
    if (i >= nx || j >= ny) return;
    const Cell c = index_cell(rho, i, j, k, nx, ny, nz, K);
    out[(static_cast<size_t>(k) * ny + j) * nx + i] = make_float4(c.dn, c.gx, c.gy, c.gz);
}

// Pass 1 of the FP16 build: max|dn| and max|g| over the grid, as the bit
// patterns of non-negative floats (ordered like unsigned integers).
__global__ void __launch_bounds__(256) field_max_kernel(const float* __restrict__ rho, int nx,
                                                        int ny, int nz, float K,
                                                        unsigned* __restrict__ max_bits) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    float mn = 0.0f, mg = 0.0f;
    if (i < nx && j < ny) {
        const Cell c = index_cell(rho, i, j, k, nx, ny, nz, K);
        mn = fabsf(c.dn);
        mg = fmaxf(fabsf(c.gx), fmaxf(fabsf(c.gy), fabsf(c.gz)));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = fmaxf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mg = fmaxf(mg, __shfl_xor_sync(0xffffffffu, mg, o));
    }
    __shared__ float sn[8], sg[8];
    const int warp = threadIdx.y;  // blockDim = (32, 8): one warp per row
    if (threadIdx.x == 0) {
        sn[warp] = mn;
        sg[warp] = mg;
    }
    __syncthreads();
    if (warp == 0 && threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) {
            mn = fmaxf(mn, sn[w]);
            mg = fmaxf(mg, sg[w]);
        }
        atomicMax(max_bits + 0, __float_as_uint(mn));
        atomicMax(max_bits + 1, __float_as_uint(mg));
    }
}

__device__ __forceinline__ float scale_of(unsigned bits) {
    const float m = __uint_as_float(bits);
    return m > 0.0f ? m / HH_FP16_CODE_MAX : 1.0f;
}

// Pass 2 of the FP16 build: quantise {dn, g} to halves with the scales.
__global__ void __launch_bounds__(256) field_fp16_kernel(const float* __restrict__ rho, int nx,
                                                         int ny, int nz, float K,
                                                         const unsigned* __restrict__ max_bits,
                                                         ushort4* __restrict__ out,
                                                         float* __restrict__ scales) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    const float s_n = scale_of(max_bits[0]);
    const float s_g = scale_of(max_bits[1]);
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
        threadIdx.y == 0) {
        scales[0] = s_n;
        scales[1] = s_g;
    }
    if (i >= nx || j >= ny) return;
    const Cell c = index_cell(rho, i, j, k, nx, ny, nz, K);
    ushort4 q;
    q.x = __half_as_ushort(__float2half_rn(c.dn / s_n));
    q.y = __half_as_ushort(__float2half_rn(c.gx / s_g));
    q.z = __half_as_ushort(__float2half_rn(c.gy / s_g));
    q.w = __half_as_ushort(__float2half_rn(c.gz / s_g));
    out[(static_cast<size_t>(k) * ny + j) * nx + i] = q;
}

__global__ void export_kernel(const void* __restrict__ data, int storage, size_t nvox,
                              const float* __restrict__ scales, float4* __restrict__ dst) {
    const size_t v = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    if (storage == HH_STORE_FP32) {
        dst[v] = reinterpret_cast<const float4*>(data)[v];
    } else {
        const ushort4 q = reinterpret_cast<const ushort4*>(data)[v];
        const float s_n = scales[0], s_g = scales[1];
        dst[v] = make_float4(__half2float(__ushort_as_half(q.x)) * s_n,
                             __half2float(__ushort_as_half(q.y)) * s_g,
                             __half2float(__ushort_as_half(q.z)) * s_g,
                             __half2float(__ushort_as_half(q.w)) * s_g);
    }
}

}  // namespace

cudaError_t launch_field(const float* rho, int nx, int ny, int nz, float K, hh_volume_s* vol,
                         cudaStream_t s) {
    const dim3 block(32, 8);
    const dim3 grid((nx + 31) / 32, (ny + 7) / 8, nz);
    if (vol->storage == HH_STORE_FP32) {
        field_fp32_kernel<<<grid, block, 0, s>>>(rho, nx, ny, nz, K,
                                                 static_cast<float4*>(vol->data),
                                                 vol->scales_dev);
        count_launch();
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(vol->max_dev, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    field_max_kernel<<<grid, block, 0, s>>>(rho, nx, ny, nz, K, vol->max_dev);
    field_fp16_kernel<<<grid, block, 0, s>>>(rho, nx, ny, nz, K, vol->max_dev,
                                             static_cast<ushort4*>(vol->data), vol->scales_dev);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_export(const hh_volume_s* vol, float4* dst, cudaStream_t s) {
    const size_t nvox = static_cast<size_t>(vol->nx) * vol->ny * vol->nz;
    const int threads = 256;
    const size_t blocks = (nvox + threads - 1) / threads;
    export_kernel<<<static_cast<unsigned>(blocks), threads, 0, s>>>(vol->data, vol->storage, nvox,
                                                                    vol->scales_dev, dst);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hh
