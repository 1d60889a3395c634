// Refractive-index volume from density (Sec. 3.3.1 of arXiv 2603.02048):
// Gladstone-Dale dn = n - 1 = K rho (Eq. 12) and g = grad n = K grad rho
// (Eq. 13) by finite differences: central inside, one-sided on the first and
// last voxel of each axis. Packed per voxel as {dn, gx, gy, gz}:
//   FP32: float4, 16 B/voxel (one pass: read rho, write the volume);
//   FP16: four halves, 8 B/voxel, dn / s_n and g / s_g with per-volume scales
//         s = the smallest power of two with max|.| / s <= 16384 (pass 1
//         reduces the maxima, pass 2 recomputes the differences and quantises
//         with exact multiplications by 1 / s; rho is read twice, nothing else
//         stored).
// Threads map to (x, y) columns, x fastest (a warp is 32 consecutive
// columns), and walk 16 z slices each, so every load of rho is coalesced, the
// z neighbours come from registers and the x/y neighbours from L1.
// The packed volume is written in the volume's layout (BRICK2 with its halo
// of edge copies for volumes the march reads, LINEAR for the allocation-free
// build's caller buffer); in BRICK2 the x-pairs of a warp land in whole
// 32-byte sectors. The volume stores are marked evict-first (st.global.cs):
// the volume outgrows L2 anyway, and this keeps the density, which the
// kernel is still reading, resident in L2 instead.
// BRICK2 builds also leave the volume's free-corner mask (the march skips the
// eight loads of a sample whose corners are all zero): the store pass records
// per column and run which slices hold a nonzero stored voxel (a 32-bit word,
// no atomics), and free_mask_kernel turns those into one bit per stored
// voxel, set when the eight voxels of the cell it is the first corner of are
// all zero. The store passes walk their runs unrolled by 2, not 4: with the
// column's bits to carry, 4 spilled and was slower.
#include "hh_internal.h"

namespace hh {
namespace {

struct Cell {
    float dn, gx, gy, gz;
};

struct OutLayout {
    int layout;
    unsigned bx, bxy;
    uint32_t* colbits;    // BRICK2: per stored (padded) column and z run, the slices
                          // where it stored a nonzero voxel (null: none); rows of
                          // `pitch` columns
    int pitch;
};

// Element of grid voxel (i, j, k) in the output layout (BRICK2: halo offset).
__device__ __forceinline__ size_t out_index(const OutLayout& L, int i, int j, int k, int nx,
                                            int ny) {
    if (L.layout == HH_LAYOUT_BRICK2) return brick2_offset(i + 1, j + 1, k + 1, L.bx, L.bxy);
    return (static_cast<size_t>(k) * ny + j) * nx + i;
}

// Scale of a channel group from the bit pattern of its maximum |value| m:
// the smallest power of two s with m / s <= HH_FP16_CODE_MAX (the largest code
// lies in (HH_FP16_CODE_MAX / 2, HH_FP16_CODE_MAX]); 1 for an all-zero group.
// A power of two makes value / s exact, a multiplication by 1 / s.
__device__ __forceinline__ float scale_of(unsigned bits) {
    const float m = __uint_as_float(bits);
    if (!(m > 0.0f)) return 1.0f;
    unsigned b = __float_as_uint(m * (1.0f / HH_FP16_CODE_MAX));  // exact: a power of two
    if (b < 0x00800000u) return __uint_as_float(0x00800000u);    // below FLT_MIN: FLT_MIN
    if (b & 0x007FFFFFu) b = (b & 0xFF800000u) + 0x00800000u;     // round up to a power of two
    return __uint_as_float(b);
}

// Column variant: each thread owns one (i, j) column and walks a run of
// FIELD_ZRUN slices, keeping rho at k-1, k, k+1 in registers, so rho is read
// from memory about once per voxel plus the four x/y neighbours (L1 hits).
#define FIELD_ZRUN 16

// 8 resident blocks of 256 threads for every mode (32 registers); the FP16
// store pass with 5 (48 registers) was 6-8 % slower, and with 6 or 7 it
// spilled more, not less.
template <int MODE>  // 0: FP32 store, 1: FP16 max pass, 2: FP16 store
__global__ void __launch_bounds__(256, 8) field_column_kernel(const float* __restrict__ rho, int nx,
                                                           int ny, int nz, float K, OutLayout L,
                                                           void* __restrict__ out,
                                                           unsigned* __restrict__ max_bits,
                                                           float* __restrict__ scales) {
    // Threads cover the stored (x, y) columns (I, J), x fastest, 256 per block
    // (a warp is 32 consecutive columns, wrapping across rows). With the
    // BRICK2 halo (h = 1, stores only) every stored column, halo included, is
    // written by its own thread with the values of grid column (clamp(I - 1),
    // clamp(J - 1)), the halo's copy of the nearest edge column; the z halo
    // slices repeat the first and last grid slice.
    const int h = (MODE != 1 && L.layout == HH_LAYOUT_BRICK2) ? 1 : 0;
    const int W = nx + 2 * h, Hh = ny + 2 * h;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int J = t / W, I = t - J * W;
    const int k0 = blockIdx.y * FIELD_ZRUN;
    const int k1 = min(k0 + FIELD_ZRUN, nz);
    float s_n = 1.0f, s_g = 1.0f;
    if (MODE == 2) {
        s_n = scale_of(max_bits[0]);
        s_g = scale_of(max_bits[1]);
    }
    const float rs_n = 1.0f / s_n, rs_g = 1.0f / s_g;  // exact: powers of two
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && MODE != 1) {
        scales[0] = s_n;
        scales[1] = s_g;
    }
    float mn = 0.0f, mg = 0.0f;
    // occupancy (the store passes): bit k - k0 set when this column stored a
    // nonzero voxel at grid slice k (padded k + 1; the halo slices repeat
    // slices 0 and nz - 1)
    constexpr bool OCC = MODE != 1;
    unsigned nzk = 0;
    if (J < Hh) {
        const int i = min(max(I - h, 0), nx - 1), j = min(max(J - h, 0), ny - 1);
        const size_t sy = nx, sz = static_cast<size_t>(nx) * ny;
        const float* col = rho + static_cast<size_t>(j) * sy + i;
        const bool xl = i > 0, xh = i < nx - 1, yl = j > 0, yh = j < ny - 1;
        float dprev = k0 > 0 ? K * __ldg(col + (k0 - 1) * sz) : 0.0f;
        float dcur = K * __ldg(col + k0 * sz);
#pragma unroll(MODE == 1 ? 4 : 2)
        for (int k = k0; k < k1; ++k) {
            const float* c = col + k * sz;
            const float dnext = (k + 1 < nz) ? K * __ldg(c + sz) : 0.0f;
            const float dxl = xl ? K * __ldg(c - 1) : 0.0f, dxh = xh ? K * __ldg(c + 1) : 0.0f;
            const float dyl = yl ? K * __ldg(c - sy) : 0.0f, dyh = yh ? K * __ldg(c + sy) : 0.0f;
            Cell e;
            e.dn = dcur;
            e.gx = !xl ? dxh - dcur : (!xh ? dcur - dxl : (dxh - dxl) * 0.5f);
            e.gy = !yl ? dyh - dcur : (!yh ? dcur - dyl : (dyh - dyl) * 0.5f);
            e.gz = (k == 0) ? dnext - dcur : (k == nz - 1 ? dcur - dprev : (dnext - dprev) * 0.5f);
            const size_t o = h ? brick2_offset(I, J, k + 1, L.bx, L.bxy)
                               : (static_cast<size_t>(k) * ny + j) * nx + i;
            // z halo copies of the first and last slice
            const bool zh = h && (k == 0 || k == nz - 1);
            const size_t oh = zh ? brick2_offset(I, J, k == 0 ? 0 : nz + 1, L.bx, L.bxy) : 0;
            bool nonzero = false;
            if (MODE == 0) {
                const float4 v = make_float4(e.dn, e.gx, e.gy, e.gz);
                __stcs(static_cast<float4*>(out) + o, v);
                if (zh) __stcs(static_cast<float4*>(out) + oh, v);
                nonzero = v.x != 0.0f || v.y != 0.0f || v.z != 0.0f || v.w != 0.0f;
            } else if (MODE == 1) {
                mn = fmaxf(mn, fabsf(e.dn));
                mg = fmaxf(mg, fmaxf(fabsf(e.gx), fmaxf(fabsf(e.gy), fabsf(e.gz))));
            } else {
                ushort4 q;  // the nearest half of value / s (exact products: s is a power of two)
                q.x = __half_as_ushort(__float2half_rn(e.dn * rs_n));
                q.y = __half_as_ushort(__float2half_rn(e.gx * rs_g));
                q.z = __half_as_ushort(__float2half_rn(e.gy * rs_g));
                q.w = __half_as_ushort(__float2half_rn(e.gz * rs_g));
                const uint2 w = make_uint2(static_cast<unsigned>(q.x) | (static_cast<unsigned>(q.y) << 16),
                                           static_cast<unsigned>(q.z) | (static_cast<unsigned>(q.w) << 16));
                __stcs(static_cast<uint2*>(out) + o, w);
                if (zh) __stcs(static_cast<uint2*>(out) + oh, w);
                nonzero = ((w.x | w.y) & 0x7FFF7FFFu) != 0u;  // a half other than +-0
            }
            if (OCC) nzk |= static_cast<unsigned>(nonzero) << (k - k0);  // k - k0 < 16
            dprev = dcur;
            dcur = dnext;
        }
    }
    if (OCC && L.colbits && J < Hh) {
        // one word per stored column and run (no atomics): bit t for grid
        // slice k0 + t (padded k0 + t + 1), and in the last run bit nz - k0
        // (at most 16) for the halo slice nz + 1, a copy of slice nz - 1; the
        // halo slice 0, a copy of slice 0, is bit 0 of the first run
        unsigned bits = nzk;
        if (k1 == nz) bits |= ((nzk >> (nz - 1 - k0)) & 1u) << (nz - k0);
        L.colbits[(static_cast<size_t>(blockIdx.y) * Hh + J) * L.pitch + I] = bits;
    }
    if (MODE == 1) {  // block maximum, then one atomic per block
        for (int o = 16; o > 0; o >>= 1) {
            mn = fmaxf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mg = fmaxf(mg, __shfl_xor_sync(0xffffffffu, mg, o));
        }
        __shared__ float sn[8], sg[8];
        if ((threadIdx.x & 31) == 0) {
            sn[threadIdx.x >> 5] = mn;
            sg[threadIdx.x >> 5] = mg;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < 8; ++w) {
                mn = fmaxf(mn, sn[w]);
                mg = fmaxf(mg, sg[w]);
            }
            atomicMax(max_bits + 0, __float_as_uint(mn));
            atomicMax(max_bits + 1, __float_as_uint(mg));
        }
    }
}

// The free-corner mask from the store pass's column words: one bit per
// stored element of the BRICK2 layout (bit b & 7 of byte b >> 3 for element
// b, i.e. a byte per brick, bit = slot), set when the voxel at padded (I, J,
// K) and its +1 neighbours on each axis (the eight corners of the trilinear
// cell whose first corner it is) hold no stored nonzero value. A thread takes
// the bricks (bx, by, bz) of one brick column (bx, by) whose slices lie in
// run r: bz = 8r + 1 .. 8r + 8 (padded slices 16r + 2 .. 16r + 17), and bz =
// 0 too when r = 0. It reads the column words of the 3 x 3 stored columns
// I = 2bx .. 2bx + 2, J = 2by .. 2by + 2 for runs r and r + 1 (zero beyond the
// stored columns and runs), shifted so that bit j stands for padded slice
// 16r + j (bit 0 only needed for r = 0: the halo slice 0), ORs neighbouring
// columns and rows for the four (x, y) slot parities and neighbouring slices
// for z, and stores each brick's byte (one writer per byte, no atomics).
__global__ void free_mask_kernel(const uint32_t* __restrict__ colbits, int pitch, int H, int runs,
                                 unsigned nbx, unsigned nby, unsigned nbz,
                                 uint8_t* __restrict__ fr) {
    const unsigned bx = blockIdx.x * 32 + threadIdx.x;
    const unsigned by = blockIdx.y * blockDim.y + threadIdx.y;
    const int r = static_cast<int>(blockIdx.z);
    if (bx >= nbx || by >= nby) return;
    unsigned xo[3][2];  // per row: columns (2bx, 2bx+1) and (2bx+1, 2bx+2) ORed
#pragma unroll
    for (int jr = 0; jr < 3; ++jr) {
        const int J = 2 * static_cast<int>(by) + jr;
        unsigned c[3] = {0u, 0u, 0u};
        if (J < H) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (r + q >= runs) break;
                const uint32_t* row = colbits + (static_cast<size_t>(r + q) * H + J) * pitch;
#pragma unroll
                for (int ic = 0; ic < 3; ++ic) {
                    const unsigned I = 2 * bx + static_cast<unsigned>(ic);
                    if (I < static_cast<unsigned>(pitch)) {
                        const unsigned w = __ldg(row + I);
                        // run r: bit t -> padded 16r + 1 + t; run r + 1: 16r + 17 + t
                        c[ic] |= q == 0 ? (w << 1) | (r == 0 ? (w & 1u) : 0u) : (w << 17);
                    }
                }
            }
        }
        xo[jr][0] = c[0] | c[1];
        xo[jr][1] = c[1] | c[2];
    }
    unsigned busy[2][2];  // [y parity][x parity]: bit j, slice 16r + j or 16r + j + 1 occupied
#pragma unroll
    for (int sy = 0; sy < 2; ++sy)
#pragma unroll
        for (int sx = 0; sx < 2; ++sx) {
            const unsigned o = xo[sy][sx] | xo[sy + 1][sx];
            busy[sy][sx] = o | (o >> 1);
        }
    const size_t nbxy = static_cast<size_t>(nbx) * nby;
    const size_t col = static_cast<size_t>(by) * nbx + bx;
    for (int m = (r == 0) ? 0 : 1; m <= 8; ++m) {
        const unsigned bz = 8u * static_cast<unsigned>(r) + static_cast<unsigned>(m);
        if (bz >= nbz) break;
        unsigned byte = 0;
#pragma unroll
        for (int sz = 0; sz < 2; ++sz)
#pragma unroll
            for (int sy = 0; sy < 2; ++sy)
#pragma unroll
                for (int sx = 0; sx < 2; ++sx)
                    byte |= ((~busy[sy][sx] >> (2 * m + sz)) & 1u) << (sx | (sy << 1) | (sz << 2));
        fr[bz * nbxy + col] = static_cast<uint8_t>(byte);
    }
}

__global__ void export_kernel(const void* __restrict__ data, int storage, OutLayout L, int nx,
                              int ny, int nz, const float* __restrict__ scales,
                              float4* __restrict__ dst) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    const int j = blockIdx.y * 8 + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= nx || j >= ny) return;
    const size_t v = (static_cast<size_t>(k) * ny + j) * nx + i;
    const size_t src = out_index(L, i, j, k, nx, ny);
    if (storage == HH_STORE_FP32) {
        dst[v] = reinterpret_cast<const float4*>(data)[src];
    } else {
        const ushort4 q = reinterpret_cast<const ushort4*>(data)[src];
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
    // 256 threads per block over the stored (x, y) columns; blockIdx.y picks
    // the z run. The FP16 max pass covers the grid columns only (no halo).
    const int h2 = vol->layout == HH_LAYOUT_BRICK2 ? 2 : 0;
    const dim3 block(256);
    const dim3 grid(static_cast<unsigned>((static_cast<int64_t>(nx + h2) * (ny + h2) + 255) / 256),
                    (nz + FIELD_ZRUN - 1) / FIELD_ZRUN);
    const dim3 grid_max(static_cast<unsigned>((static_cast<int64_t>(nx) * ny + 255) / 256),
                        (nz + FIELD_ZRUN - 1) / FIELD_ZRUN);
    const bool masks = vol->layout == HH_LAYOUT_BRICK2 && vol->colbits_dev != nullptr;
    const int pitch = (nx + 2 + 3) & ~3;
    const int runs = (nz + FIELD_ZRUN - 1) / FIELD_ZRUN;
    const OutLayout L{vol->layout, vol->bx, vol->bxy, masks ? vol->colbits_dev : nullptr, pitch};
    cudaError_t e = cudaSuccess;
    if (vol->storage == HH_STORE_FP32) {
        field_column_kernel<0><<<grid, block, 0, s>>>(rho, nx, ny, nz, K, L, vol->data, nullptr,
                                                      vol->scales_dev);
        count_launch();
    } else {
        e = cudaMemsetAsync(vol->max_dev, 0, 2 * sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        field_column_kernel<1><<<grid_max, block, 0, s>>>(rho, nx, ny, nz, K, L, nullptr,
                                                          vol->max_dev, vol->scales_dev);
        field_column_kernel<2><<<grid, block, 0, s>>>(rho, nx, ny, nz, K, L, vol->data,
                                                      vol->max_dev, vol->scales_dev);
        count_launch(2);
    }
    if (masks) {
        const unsigned nby = vol->bxy / vol->bx;
        const dim3 mblock(32, 8);
        const dim3 mgrid((vol->bx + 31) / 32, (nby + 7) / 8, static_cast<unsigned>(runs));
        free_mask_kernel<<<mgrid, mblock, 0, s>>>(vol->colbits_dev, pitch, ny + 2, runs, vol->bx,
                                                  nby, vol->bz,
                                                  reinterpret_cast<uint8_t*>(vol->free_dev));
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_export(const hh_volume_s* vol, float4* dst, cudaStream_t s) {
    const dim3 block(32, 8);
    const dim3 grid((vol->nx + 31) / 32, (vol->ny + 7) / 8, vol->nz);
    const OutLayout L{vol->layout, vol->bx, vol->bxy, nullptr, 0};
    export_kernel<<<grid, block, 0, s>>>(vol->data, vol->storage, L, vol->nx, vol->ny, vol->nz,
                                         vol->scales_dev, dst);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hh
