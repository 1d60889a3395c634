// C ABI of the curved-ray heat-haze engine (declared in include/hh.h):
// argument validation, volume handles, stream-ordered scratch (the density
// grid, and for grids larger than L2 the particles binned by cell) and error
// reporting around the kernels of splat.cu, field.cu and march.cu. The batch
// API lives with its kernel in march.cu, the frame pipeline in pipeline.cpp,
// the render server in serve.cpp.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "hh_internal.h"

namespace hh {

std::atomic<uint64_t> g_launches{0};

thread_local std::string t_last_error;

hh_status fail(hh_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return st;
}

hh_status cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a sticky-free error so later calls start clean
    return fail(e == cudaErrorMemoryAllocation ? HH_ERR_OOM : HH_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

hh_status ok() {
    t_last_error.clear();
    return HH_OK;
}

// Allocation wrappers: every device and pinned-host buffer the library owns
// goes through them, so the live count below is the library's whole
// footprint. HH_FAIL_ALLOC_AT=k makes the k-th allocation (counted from the
// last change of the variable's value) fail with cudaErrorMemoryAllocation
// without allocating, which drives each entry point's out-of-memory path on
// demand.
namespace {
std::mutex g_alloc_mutex;
std::string g_fail_spec;
long g_fail_count = 0;
std::atomic<int64_t> g_live_allocs{0};

bool injected_failure() {
    const char* spec = std::getenv("HH_FAIL_ALLOC_AT");
    if (!spec || !*spec) return false;
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    if (g_fail_spec != spec) {
        g_fail_spec = spec;
        g_fail_count = 0;
    }
    return ++g_fail_count == std::atol(spec);
}
}  // namespace

cudaError_t dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) g_live_allocs.fetch_add(1);
    else *p = nullptr;
    return e;
}

void dev_free(void* p) {
    if (!p) return;
    cudaFree(p);
    g_live_allocs.fetch_sub(1);
}

cudaError_t host_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (injected_failure()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocHost(p, bytes);
    if (e == cudaSuccess) g_live_allocs.fetch_add(1);
    else *p = nullptr;
    return e;
}

void host_free(void* p) {
    if (!p) return;
    cudaFreeHost(p);
    g_live_allocs.fetch_sub(1);
}

int64_t live_allocations() { return g_live_allocs.load(); }

namespace {

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// Largest grid the kernels index with 32-bit per-axis coordinates and
// 64-bit linear offsets.
constexpr int kMaxAxis = 1 << 14;

hh_status check_grid(const hh_grid* g, bool need_h) {
    if (!g) return fail(HH_ERR_INVALID_ARG, "grid is NULL");
    if (g->nx < 2 || g->ny < 2 || g->nz < 2 || g->nx > kMaxAxis || g->ny > kMaxAxis ||
        g->nz > kMaxAxis)
        return fail(HH_ERR_INVALID_ARG, "grid %d x %d x %d: each axis must be in [2, %d]", g->nx,
                    g->ny, g->nz, kMaxAxis);
    if (g->storage != HH_STORE_FP32 && g->storage != HH_STORE_FP16_SCALED)
        return fail(HH_ERR_INVALID_ARG, "unknown storage %d", g->storage);
    if (static_cast<size_t>(brick2_count(g->nx)) * brick2_count(g->ny) * brick2_count(g->nz) * 8 >
        (size_t(1) << 31))
        return fail(HH_ERR_INVALID_ARG, "grid %d x %d x %d: more than 2^31 stored voxels", g->nx,
                    g->ny, g->nz);
    if (need_h && !(g->h_kernel > 0.0f && std::isfinite(g->h_kernel)))
        return fail(HH_ERR_INVALID_ARG, "h_kernel must be a positive finite number");
    return HH_OK;
}

hh_status check_particles(const hh_particles* p) {
    if (!p) return fail(HH_ERR_INVALID_ARG, "particles is NULL");
    if (p->n < 0) return fail(HH_ERR_INVALID_ARG, "negative particle count");
    if (p->n > 0 && !p->xyzm_dev) return fail(HH_ERR_INVALID_ARG, "particle pointer is NULL");
    if (p->n > (int64_t(1) << 36)) return fail(HH_ERR_INVALID_ARG, "too many particles");
    if (reinterpret_cast<uintptr_t>(p->xyzm_dev) % 16 != 0)
        return fail(HH_ERR_INVALID_ARG, "particle array must be 16-byte aligned (float4)");
    return HH_OK;
}

size_t voxels(const hh_grid* g) { return static_cast<size_t>(g->nx) * g->ny * g->nz; }

hh_status new_volume(const hh_grid* g, hh_volume* out) {
    if (!out) return fail(HH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    hh_volume_s* v = new (std::nothrow) hh_volume_s();
    if (!v) return fail(HH_ERR_OOM, "host allocation failed");
    v->nx = g->nx;
    v->ny = g->ny;
    v->nz = g->nz;
    v->storage = g->storage;
    v->h_kernel = g->h_kernel;
    v->layout = HH_LAYOUT_BRICK2;
    v->bx = brick2_count(g->nx);
    v->bxy = v->bx * brick2_count(g->ny);
    const size_t padded = static_cast<size_t>(v->bxy) * brick2_count(g->nz) * 8;
    v->bytes = padded * (g->storage == HH_STORE_FP32 ? 16 : 8);
    v->bz = brick2_count(g->nz);
    v->mask_words = (padded + 31) / 32;  // one bit per element (8 per brick, a byte)
    // the free-corner mask and its build scratch (a word per stored column
    // and 16-slice z run, rows padded to 4 columns) follow the data in the
    // same allocation (the data's size is a multiple of 64 bytes, so the mask
    // is aligned); all of it starts zero: even-padding voxels read as 0, and
    // no element is marked free before the first build
    const size_t colbytes = static_cast<size_t>((g->nx + 2 + 3) & ~3) * (g->ny + 2) *
                            ((g->nz + 15) / 16) * sizeof(uint32_t);
    const size_t total = v->bytes + v->mask_words * sizeof(unsigned) + colbytes;
    cudaGetDevice(&v->device);
    cudaError_t e = dev_alloc(&v->data, total);
    if (e == cudaSuccess) e = cudaMemset(v->data, 0, total);
    if (e == cudaSuccess) {
        v->free_dev = reinterpret_cast<unsigned*>(static_cast<char*>(v->data) + v->bytes);
        v->colbits_dev = reinterpret_cast<uint32_t*>(v->free_dev + v->mask_words);
    }
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void**>(&v->scales_dev), 2 * sizeof(float));
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void**>(&v->max_dev), 2 * sizeof(unsigned));
    if (e != cudaSuccess) {
        dev_free(v->data);
        dev_free(v->scales_dev);
        dev_free(v->max_dev);
        delete v;
        return cuda_fail(e, "volume allocation");
    }
    *out = v;
    return HH_OK;
}

void drop_volume(hh_volume v) {
    if (!v) return;
    dev_free(v->rho_dev);
    dev_free(v->sorted_dev);
    dev_free(v->bins_dev);
    dev_free(v->data);
    dev_free(v->scales_dev);
    dev_free(v->max_dev);
    delete v;
}

// Whether hh_volume_rebuild sorts the particles by cell before the splat:
// when the density grid is larger than the device's L2 (so randomly ordered
// reductions would miss it) and there are enough particles to pay for the
// sort. HH_SPLAT_SORT=0 / 1 forces it off / on.
bool sort_particles(const hh_volume_s* v, int64_t n) {
    if (n <= 0 || n >= (int64_t(1) << 31)) return false;
    const char* env = std::getenv("HH_SPLAT_SORT");
    if (env && env[0] == '0') return false;
    if (env && env[0] == '1') return true;
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, v->device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const size_t rho_bytes = static_cast<size_t>(v->nx) * v->ny * v->nz * sizeof(float);
    return n >= 65536 && rho_bytes > static_cast<size_t>(l2);
}

// Grows the binning scratch of `v` to n particles (cudaMalloc, synchronous).
hh_status sort_scratch(hh_volume_s* v, int64_t n) {
    if (!v->bins_dev) {
        v->n_bins = splat_bin_count(v->nx, v->ny, v->nz);
        cudaError_t e = dev_alloc(reinterpret_cast<void**>(&v->bins_dev),
                                   2 * static_cast<size_t>(v->n_bins) * sizeof(unsigned));
        if (e != cudaSuccess) {
            v->bins_dev = nullptr;
            return cuda_fail(e, "particle binning scratch");
        }
    }
    if (v->sorted_cap < n) {
        dev_free(v->sorted_dev);
        v->sorted_dev = nullptr;
        v->sorted_cap = 0;
        cudaError_t e = dev_alloc(reinterpret_cast<void**>(&v->sorted_dev),
                                   static_cast<size_t>(n) * sizeof(float4));
        if (e != cudaSuccess) {
            v->sorted_dev = nullptr;
            return cuda_fail(e, "sorted particle scratch");
        }
        v->sorted_cap = n;
    }
    return HH_OK;
}

hh_status volume_from(const float* rho_dev, const hh_grid* grid, float K, cudaStream_t s,
                      hh_volume* out) {
    hh_volume v = nullptr;
    hh_status st = new_volume(grid, &v);
    if (st != HH_OK) return st;
    cudaError_t e = launch_field(rho_dev, grid->nx, grid->ny, grid->nz, K, v, s);
    if (e != cudaSuccess) {
        drop_volume(v);
        return cuda_fail(e, "field kernel launch");
    }
    *out = v;
    return ok();
}

}  // namespace

hh_status check_params(const hh_step_params* P) {
    if (!P) return fail(HH_ERR_INVALID_ARG, "step params is NULL");
    if (P->stepper != HH_STEP_EULER_PAPER && P->stepper != HH_STEP_RK4)
        return fail(HH_ERR_INVALID_ARG, "unknown stepper %d", P->stepper);
    if (P->max_steps < 0) return fail(HH_ERR_INVALID_ARG, "max_steps must be >= 0");
    if (P->adaptive) {
        if (!(P->h_min > 0.0f) || !(P->h_max >= P->h_min) || !std::isfinite(P->h_max))
            return fail(HH_ERR_INVALID_ARG, "adaptive step needs 0 < h_min <= h_max < inf");
        if (!(P->theta_max >= 0.0f) || !std::isfinite(P->theta_max))
            return fail(HH_ERR_INVALID_ARG, "theta_max must be finite and >= 0");
        if (!(P->eps > 0.0f) || !std::isfinite(P->eps))
            return fail(HH_ERR_INVALID_ARG, "eps must be finite and > 0");
    } else if (!(P->h_fixed > 0.0f) || !std::isfinite(P->h_fixed)) {
        return fail(HH_ERR_INVALID_ARG, "h_fixed must be finite and > 0");
    }
    return HH_OK;
}

hh_status check_background(const hh_background* bg) {
    if (!bg || !bg->rgb8_dev || bg->width < 1 || bg->height < 2)
        return fail(HH_ERR_INVALID_ARG, "background needs a device pointer, width >= 1, height >= 2");
    if (bg->n_planes < 0 || bg->n_planes > HH_MAX_PLANES)
        return fail(HH_ERR_INVALID_ARG, "n_planes must be in [0, %d]", HH_MAX_PLANES);
    for (int k = 0; k < bg->n_planes; ++k) {
        const hh_plane& p = bg->planes[k];
        if (!p.rgb8_dev || p.width < 2 || p.height < 2)
            return fail(HH_ERR_INVALID_ARG, "plane %d needs a device texture of at least 2 x 2", k);
        float uu = 0.0f, vv = 0.0f, uv = 0.0f;
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(p.origin[a]) || !std::isfinite(p.u[a]) || !std::isfinite(p.v[a]))
                return fail(HH_ERR_INVALID_ARG, "plane %d: non-finite vector", k);
            uu += p.u[a] * p.u[a];
            vv += p.v[a] * p.v[a];
            uv += p.u[a] * p.v[a];
        }
        if (!(uu > 0.0f) || !(vv > 0.0f) || std::fabs(uv) > 1e-4f * std::sqrt(uu * vv))
            return fail(HH_ERR_INVALID_ARG, "plane %d: u and v must be non-zero and perpendicular", k);
    }
    return HH_OK;
}

hh_status check_camera(const hh_camera& c, int i) {
    if (c.width < 1 || c.height < 1 || c.width > 65536 || c.height > 65536 ||
        static_cast<int64_t>(c.width) * c.height > (int64_t(1) << 31))
        return fail(HH_ERR_INVALID_ARG, "camera %d: bad resolution %d x %d", i, c.width, c.height);
    if (!(c.vfov_deg > 0.0f && c.vfov_deg < 180.0f))
        return fail(HH_ERR_INVALID_ARG, "camera %d: vfov must be in (0, 180)", i);
    float f[3], n2 = 0.0f;
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(c.eye[a]) || !std::isfinite(c.look_at[a]) || !std::isfinite(c.up[a]))
            return fail(HH_ERR_INVALID_ARG, "camera %d: non-finite vector", i);
        f[a] = c.look_at[a] - c.eye[a];
        n2 += f[a] * f[a];
    }
    const float cx = f[1] * c.up[2] - f[2] * c.up[1], cy = f[2] * c.up[0] - f[0] * c.up[2],
                cz = f[0] * c.up[1] - f[1] * c.up[0];
    if (!(n2 > 0.0f) || !(cx * cx + cy * cy + cz * cz > 0.0f))
        return fail(HH_ERR_INVALID_ARG, "camera %d: look_at == eye or up parallel to the view", i);
    return HH_OK;
}

}  // namespace hh

using namespace hh;

extern "C" {

const char* hh_last_error(void) { return t_last_error.c_str(); }

uint64_t hh_kernel_launch_count(void) { return g_launches.load(); }

int64_t hh_live_allocations(void) { return live_allocations(); }

hh_status hh_splat_density(const hh_particles* particles, const hh_grid* grid, float* rho_dev,
                           void* stream) {
    hh_status st = check_grid(grid, true);
    if (st != HH_OK) return st;
    if ((st = check_particles(particles)) != HH_OK) return st;
    if (!rho_dev) return fail(HH_ERR_INVALID_ARG, "rho_dev is NULL");
    cudaError_t e = launch_splat(reinterpret_cast<const float4*>(particles->xyzm_dev), particles->n,
                                 grid->nx, grid->ny, grid->nz, grid->h_kernel, rho_dev,
                                 as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, "splat launch");
    return ok();
}

hh_status hh_volume_from_density(const float* rho_dev, const hh_grid* grid, float K_gd,
                                 void* stream, hh_volume* out) {
    hh_status st = check_grid(grid, false);
    if (st != HH_OK) return st;
    if (!rho_dev) return fail(HH_ERR_INVALID_ARG, "rho_dev is NULL");
    if (!std::isfinite(K_gd)) return fail(HH_ERR_INVALID_ARG, "K_gd must be finite");
    return volume_from(rho_dev, grid, K_gd, as_stream(stream), out);
}

hh_status hh_volume_from_dn(const float* dn_dev, const hh_grid* grid, void* stream,
                            hh_volume* out) {
    return hh_volume_from_density(dn_dev, grid, 1.0f, stream, out);
}

hh_status hh_build_index_field(const hh_particles* particles, const hh_grid* grid, float K_gd,
                               void* stream, hh_volume* out) {
    hh_status st = check_grid(grid, true);
    if (st != HH_OK) return st;
    if ((st = check_particles(particles)) != HH_OK) return st;
    if (!std::isfinite(K_gd)) return fail(HH_ERR_INVALID_ARG, "K_gd must be finite");
    hh_volume v = nullptr;
    if ((st = new_volume(grid, &v)) != HH_OK) return st;
    cudaError_t e = dev_alloc(reinterpret_cast<void**>(&v->rho_dev), voxels(grid) * sizeof(float));
    if (e != cudaSuccess) {
        drop_volume(v);
        return cuda_fail(e, "density scratch");
    }
    if ((st = hh_volume_rebuild(v, particles, K_gd, stream)) != HH_OK) {
        drop_volume(v);
        return st;
    }
    *out = v;
    return ok();
}

hh_status hh_volume_rebuild(hh_volume vol, const hh_particles* particles, float K_gd,
                            void* stream) {
    if (!vol) return fail(HH_ERR_INVALID_ARG, "volume is NULL");
    hh_status st = check_particles(particles);
    if (st != HH_OK) return st;
    if (!std::isfinite(K_gd)) return fail(HH_ERR_INVALID_ARG, "K_gd must be finite");
    if (!(vol->h_kernel > 0.0f && std::isfinite(vol->h_kernel)))
        return fail(HH_ERR_INVALID_ARG, "volume has no splat kernel radius (h_kernel <= 0)");
    const size_t nvox = static_cast<size_t>(vol->nx) * vol->ny * vol->nz;
    if (!vol->rho_dev) {
        cudaError_t e = dev_alloc(reinterpret_cast<void**>(&vol->rho_dev), nvox * sizeof(float));
        if (e != cudaSuccess) {
            vol->rho_dev = nullptr;
            return cuda_fail(e, "density scratch");
        }
    }
    cudaStream_t s = as_stream(stream);
    const float4* src = reinterpret_cast<const float4*>(particles->xyzm_dev);
    if (sort_particles(vol, particles->n)) {
        if ((st = sort_scratch(vol, particles->n)) != HH_OK) return st;
        cudaError_t e = launch_bin_particles(src, particles->n, vol->nx, vol->ny, vol->nz,
                                             vol->bins_dev, vol->sorted_dev, s);
        if (e != cudaSuccess) return cuda_fail(e, "particle binning launch");
        src = vol->sorted_dev;
    }
    cudaError_t e = launch_splat(src, particles->n, vol->nx, vol->ny, vol->nz, vol->h_kernel,
                                 vol->rho_dev, s);
    if (e != cudaSuccess) return cuda_fail(e, "splat launch");
    e = launch_field(vol->rho_dev, vol->nx, vol->ny, vol->nz, K_gd, vol, s);
    if (e != cudaSuccess) return cuda_fail(e, "field kernel launch");
    return ok();
}

hh_status hh_volume_export(hh_volume vol, float* dst_dev, void* stream) {
    if (!vol || !dst_dev) return fail(HH_ERR_INVALID_ARG, "volume or destination is NULL");
    if (reinterpret_cast<uintptr_t>(dst_dev) % 16 != 0)
        return fail(HH_ERR_INVALID_ARG, "destination must be 16-byte aligned");
    cudaError_t e = launch_export(vol, reinterpret_cast<float4*>(dst_dev), as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, "export launch");
    return ok();
}

hh_status hh_volume_info(hh_volume vol, hh_grid* grid, float* s_n, float* s_g, size_t* bytes,
                         void* stream) {
    if (!vol) return fail(HH_ERR_INVALID_ARG, "volume is NULL");
    if (grid) {
        grid->nx = vol->nx;
        grid->ny = vol->ny;
        grid->nz = vol->nz;
        grid->h_kernel = vol->h_kernel;
        grid->storage = vol->storage;
    }
    if (bytes) *bytes = vol->bytes;
    if (s_n || s_g) {
        float sc[2];
        cudaError_t e = cudaMemcpyAsync(sc, vol->scales_dev, sizeof sc, cudaMemcpyDeviceToHost,
                                        as_stream(stream));
        if (e == cudaSuccess) e = cudaStreamSynchronize(as_stream(stream));
        if (e != cudaSuccess) return cuda_fail(e, "reading volume scales");
        if (s_n) *s_n = sc[0];
        if (s_g) *s_g = sc[1];
    }
    return ok();
}

hh_status hh_volume_scales(hh_volume vol, float* s_n, float* s_g) {
    return hh_volume_info(vol, nullptr, s_n, s_g, nullptr, nullptr);
}

hh_status hh_volume_free(hh_volume vol) {
    if (!vol) return ok();
    cudaError_t e = cudaDeviceSynchronize();
    drop_volume(vol);
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before volume free");
    return ok();
}

hh_status hh_trace(hh_volume vol, const hh_camera* cams, int n_cams,
                   const hh_step_params* params, const hh_background* bg,
                   const hh_view_out* outs, void* stream) {
    if (!vol) return fail(HH_ERR_INVALID_ARG, "volume is NULL");
    if (n_cams < 0) return fail(HH_ERR_INVALID_ARG, "negative camera count");
    if (n_cams > 0 && (!cams || !outs)) return fail(HH_ERR_INVALID_ARG, "cameras/outputs NULL");
    hh_status st = check_params(params);
    if (st != HH_OK) return st;
    if ((st = check_background(bg)) != HH_OK) return st;
    for (int i = 0; i < n_cams; ++i) {
        if ((st = check_camera(cams[i], i)) != HH_OK) return st;
        if (!outs[i].rgb && !outs[i].rgb8)
            return fail(HH_ERR_INVALID_ARG, "view %d: rgb and rgb8 outputs are both NULL", i);
    }
    for (int i = 0; i < n_cams; ++i) {
        cudaError_t e = launch_trace(vol, cams[i], *params, *bg, outs[i], as_stream(stream));
        if (e != cudaSuccess) return cuda_fail(e, "march launch");
    }
    return ok();
}

}  // extern "C"
