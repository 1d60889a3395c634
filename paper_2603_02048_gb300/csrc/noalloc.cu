// Allocation-free variant of the volume build (hh_build_index_field_noalloc).
//
// Some callers cannot allocate device memory at all: a host application that
// owns the whole device-memory budget and forbids libraries from allocating
// (engine or plugin hosts with a fixed pool), or a real-time frame loop that
// must not pay cudaMalloc's implicit device synchronisation and unbounded
// latency. For them the density grid that the splat accumulates into lives in
// a file-scope device array of fixed size instead of a cudaMalloc'ed buffer;
// the caller passes the particles in and the packed FP32 {dn, grad n} volume
// buffer out, and nothing is allocated.
//
// The array costs HH_NOALLOC_MAX_VOXELS * 4 bytes (8 MiB) on every device that
// loads the library, until the process exits. Host code cannot use the
// array's name as a device address (in host code it names a host-side stand-in),
// so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call there.
#include <mutex>

#include "hh_internal.h"

#define HH_NOALLOC_MAX_VOXELS (1u << 21)  // 2,097,152 voxels, e.g. 128^3
#define HH_NOALLOC_MAX_DEVICES 64

namespace {

// Shared by every call on a device; each call overwrites it (the density is
// cleared at the start of every call).
static __device__ __align__(256) float g_noalloc_rho[HH_NOALLOC_MAX_VOXELS];
static __device__ __align__(256) float g_noalloc_scales[2];
static __device__ __align__(256) unsigned g_noalloc_max[2];

struct StaticScratch {
    bool ready = false;
    float* rho = nullptr;
    float* scales = nullptr;
    unsigned* max = nullptr;
};

std::mutex g_setup_mutex;
StaticScratch g_scratch[HH_NOALLOC_MAX_DEVICES];

// Device addresses of the static arrays on the current device (once per device).
hh_status static_scratch(StaticScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return hh::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= HH_NOALLOC_MAX_DEVICES)
        return hh::fail(HH_ERR_INVALID_ARG, "device ordinal %d is beyond %d", dev,
                        HH_NOALLOC_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    StaticScratch& s = g_scratch[dev];
    if (!s.ready) {
        e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.rho), g_noalloc_rho);
        if (e == cudaSuccess)
            e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.scales), g_noalloc_scales);
        if (e == cudaSuccess)
            e = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.max), g_noalloc_max);
        if (e != cudaSuccess) return hh::cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
        s.ready = true;
    }
    *out = &s;
    return HH_OK;
}

}  // namespace

extern "C" hh_status hh_build_index_field_noalloc(const hh_particles* particles,
                                                  const hh_grid* grid, float K_gd,
                                                  float* vol4_dev, void* stream) {
    if (!particles || !grid) return hh::fail(HH_ERR_INVALID_ARG, "particles or grid is NULL");
    if (grid->nx < 2 || grid->ny < 2 || grid->nz < 2)
        return hh::fail(HH_ERR_INVALID_ARG, "grid %d x %d x %d: each axis must be >= 2", grid->nx,
                        grid->ny, grid->nz);
    const size_t nvox = static_cast<size_t>(grid->nx) * grid->ny * grid->nz;
    if (nvox > HH_NOALLOC_MAX_VOXELS)
        return hh::fail(HH_ERR_INVALID_ARG,
                        "grid %d x %d x %d has %zu voxels; the allocation-free build holds at "
                        "most %u (use hh_build_index_field for larger grids)",
                        grid->nx, grid->ny, grid->nz, nvox, HH_NOALLOC_MAX_VOXELS);
    if (grid->storage != HH_STORE_FP32)
        return hh::fail(HH_ERR_INVALID_ARG, "the allocation-free build writes FP32 storage only");
    if (!(grid->h_kernel > 0.0f && grid->h_kernel < 1e30f))
        return hh::fail(HH_ERR_INVALID_ARG, "h_kernel must be a positive finite number");
    if (!(K_gd == K_gd) || K_gd > 1e30f || K_gd < -1e30f)
        return hh::fail(HH_ERR_INVALID_ARG, "K_gd must be finite");
    if (particles->n < 0 || (particles->n > 0 && !particles->xyzm_dev) ||
        reinterpret_cast<uintptr_t>(particles->xyzm_dev) % 16 != 0)
        return hh::fail(HH_ERR_INVALID_ARG, "particles must be a 16-byte aligned float4 array");
    if (!vol4_dev || reinterpret_cast<uintptr_t>(vol4_dev) % 16 != 0)
        return hh::fail(HH_ERR_INVALID_ARG, "vol4_dev must be a 16-byte aligned device buffer");

    StaticScratch* s = nullptr;
    hh_status st = static_scratch(&s);
    if (st != HH_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    // launch_splat clears the density (cudaMemsetAsync) before accumulating.
    cudaError_t e = hh::launch_splat(reinterpret_cast<const float4*>(particles->xyzm_dev),
                                     particles->n, grid->nx, grid->ny, grid->nz, grid->h_kernel,
                                     s->rho, cs);
    if (e != cudaSuccess) return hh::cuda_fail(e, "splat launch");
    hh_volume_s out{};
    out.nx = grid->nx;
    out.ny = grid->ny;
    out.nz = grid->nz;
    out.storage = HH_STORE_FP32;
    out.layout = HH_LAYOUT_LINEAR;  // the documented x-fastest output
    out.h_kernel = grid->h_kernel;
    out.data = vol4_dev;
    out.bytes = nvox * 16;
    out.scales_dev = s->scales;
    out.max_dev = s->max;
    e = hh::launch_field(s->rho, grid->nx, grid->ny, grid->nz, K_gd, &out, cs);
    if (e != cudaSuccess) return hh::cuda_fail(e, "field kernel launch");
    return hh::ok();
}
