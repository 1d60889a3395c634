// Real-time frame pipeline (hh_pipeline_*): per simulation frame, particles
// from host memory are splatted into the volume (Sec. 3.3.1) and every view
// is marched through it (Secs. 3.3.2-3.3.3), and the display images go back
// to host memory.
//
// Frames alternate between two slots, each with its own volume, device
// particle buffer, image buffers, events and two compute streams: `up`
// copies a frame's particles to the device, the slot's `build` stream
// rebuilds the slot's volume, its `march` stream marches the views, `down`
// copies the images back. With a volume per slot, frame t+1's splat and
// field kernels run beside frame t's march; their stream has the device's
// highest priority, so their blocks take the SMs as the march's blocks
// retire (the build's memory-bound field pass fills the march's issue gaps)
// instead of waiting for the whole march. The upload of frame t+1 and the
// download of frame t-1 run on the copy engines meanwhile. Submitting frame t first waits for frame t-2 (the
// slot's previous frame) to complete, which bounds the frames in flight to
// two. All host waits are bounded.
#include <algorithm>
#include <chrono>
#include <thread>
#include <vector>

#include "hh_internal.h"

namespace {

constexpr int kSlots = 2;
constexpr int kMaxViews = 4096;
constexpr int kSubmitWaitMs = 60000;

struct PipeSlot {
    hh_volume vol = nullptr;         // this slot's frames' volume
    cudaStream_t build = nullptr;    // rebuild of this slot's frames (highest priority)
    cudaStream_t march = nullptr;    // march of this slot's frames
    float* parts_dev = nullptr;      // max_particles float4
    uint8_t* rgb8_dev = nullptr;     // every view's H*W*3 bytes, back to back
    std::vector<hh_view_out> outs;   // rgb8 pointers into rgb8_dev
    hh_batch batch = nullptr;        // the views as one launch (cfg given)
    cudaEvent_t uploaded = nullptr, built = nullptr, rendered = nullptr, downloaded = nullptr;
    int64_t frame = -1;              // last frame submitted in this slot
};

// Waits for `ev` with a bound (polling: yields for the first 2 ms, then
// sleeps 50 us between queries); cudaErrorNotReady once the bound passes.
cudaError_t wait_event(cudaEvent_t ev, int timeout_ms) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t q = cudaEventQuery(ev);
        if (q != cudaErrorNotReady) return q;
        const auto us = std::chrono::duration_cast<std::chrono::microseconds>(
                            std::chrono::steady_clock::now() - t0)
                            .count();
        if (us >= static_cast<long long>(timeout_ms) * 1000) return cudaErrorNotReady;
        if (us < 2000)
            std::this_thread::yield();
        else
            std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// Makes `device` current for the scope and restores the caller's device.
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != device) cudaSetDevice(device);
    }
    ~DeviceScope() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

struct hh_pipeline_s {
    float K = 0.0f;
    int64_t max_particles = 0;
    std::vector<hh_camera> cams;
    std::vector<size_t> view_bytes;  // H*W*3 per view
    hh_step_params params{};
    hh_background bg{};
    bool batched = false;
    cudaStream_t up = nullptr, down = nullptr;
    PipeSlot slot[kSlots];
    uint64_t next_frame = 0;
    int device = 0;

    ~hh_pipeline_s() {
        for (PipeSlot& s : slot) {
            if (s.batch) hh_batch_free(s.batch);
            hh::dev_free(s.parts_dev);
            hh::dev_free(s.rgb8_dev);
            if (s.uploaded) cudaEventDestroy(s.uploaded);
            if (s.rendered) cudaEventDestroy(s.rendered);
            if (s.downloaded) cudaEventDestroy(s.downloaded);
            if (s.built) cudaEventDestroy(s.built);
            if (s.vol) hh_volume_free(s.vol);
            if (s.build) cudaStreamDestroy(s.build);
            if (s.march) cudaStreamDestroy(s.march);
        }
        if (up) cudaStreamDestroy(up);
        if (down) cudaStreamDestroy(down);
    }
};

extern "C" {

hh_status hh_pipeline_create(const hh_grid* grid, float K_gd, int64_t max_particles,
                             const hh_camera* cams, int n_cams, const hh_step_params* params,
                             const hh_background* bg, const hh_batch_config* cfg,
                             hh_pipeline* out) {
    using hh::fail;
    if (!out) return fail(HH_ERR_INVALID_ARG, "output handle pointer is NULL");
    *out = nullptr;
    if (!grid) return fail(HH_ERR_INVALID_ARG, "grid is NULL");
    if (max_particles < 0 || max_particles > (int64_t(1) << 36))
        return fail(HH_ERR_INVALID_ARG, "max_particles out of range");
    if (n_cams < 1 || n_cams > kMaxViews || !cams)
        return fail(HH_ERR_INVALID_ARG, "need 1..%d cameras", kMaxViews);
    hh_status st = hh::check_params(params);
    if (st != HH_OK) return st;
    if ((st = hh::check_background(bg)) != HH_OK) return st;
    for (int i = 0; i < n_cams; ++i)
        if ((st = hh::check_camera(cams[i], i)) != HH_OK) return st;

    hh_pipeline p = new hh_pipeline_s();
    p->K = K_gd;
    p->max_particles = max_particles;
    p->cams.assign(cams, cams + n_cams);
    p->params = *params;
    p->bg = *bg;
    p->batched = cfg != nullptr;
    cudaGetDevice(&p->device);
    size_t total = 0;
    for (const hh_camera& c : p->cams) {
        p->view_bytes.push_back(static_cast<size_t>(c.width) * c.height * 3);
        total += (p->view_bytes.back() + 255) & ~size_t(255);
    }
    cudaError_t e = cudaSuccess;
    for (cudaStream_t* s : {&p->up, &p->down, &p->slot[0].march, &p->slot[1].march})
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    for (PipeSlot& s : p->slot)
        if (e == cudaSuccess)
            e = cudaStreamCreateWithPriority(&s.build, cudaStreamNonBlocking, greatest);
    if (e != cudaSuccess) {
        delete p;
        return hh::cuda_fail(e, "pipeline streams");
    }
    // the slots' volumes, built empty once (allocates them and their density scratch)
    const hh_particles none{nullptr, 0};
    for (PipeSlot& s : p->slot)
        if ((st = hh_build_index_field(&none, grid, K_gd, s.build, &s.vol)) != HH_OK) {
            delete p;
            return st;
        }
    for (PipeSlot& s : p->slot) {
        e = hh::dev_alloc(reinterpret_cast<void**>(&s.parts_dev),
                       static_cast<size_t>(std::max<int64_t>(max_particles, 1)) * 16);
        if (e == cudaSuccess) e = hh::dev_alloc(reinterpret_cast<void**>(&s.rgb8_dev), total);
        for (cudaEvent_t* ev : {&s.uploaded, &s.built, &s.rendered, &s.downloaded})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            delete p;
            return hh::cuda_fail(e, "pipeline buffers");
        }
        size_t off = 0;
        for (size_t v = 0; v < p->cams.size(); ++v) {
            hh_view_out o{};
            o.rgb8 = s.rgb8_dev + off;
            s.outs.push_back(o);
            off += (p->view_bytes[v] + 255) & ~size_t(255);
        }
        if (p->batched) {
            if ((st = hh_batch_create(s.vol, cams, n_cams, params, bg, s.outs.data(),
                                      &s.batch)) != HH_OK ||
                (st = hh_batch_set_config(s.batch, cfg)) != HH_OK) {
                delete p;
                return st;
            }
        }
    }
    for (PipeSlot& s : p->slot) {
        if (e == cudaSuccess) e = cudaEventRecord(s.rendered, s.build);
        if (e == cudaSuccess) e = wait_event(s.rendered, kSubmitWaitMs);
    }
    if (e != cudaSuccess) {
        delete p;
        return e == cudaErrorNotReady ? fail(HH_ERR_TIMEOUT, "pipeline set-up timed out")
                                      : hh::cuda_fail(e, "pipeline set-up");
    }
    *out = p;
    return hh::ok();
}

hh_status hh_pipeline_submit(hh_pipeline p, const float* xyzm_host, int64_t n,
                             uint8_t* const* rgb8_host, uint64_t* frame) {
    using hh::fail;
    if (!p) return fail(HH_ERR_INVALID_ARG, "pipeline is NULL");
    if (n < 0 || n > p->max_particles)
        return fail(HH_ERR_INVALID_ARG, "particle count %lld outside [0, %lld]",
                    static_cast<long long>(n), static_cast<long long>(p->max_particles));
    if (n > 0 && !xyzm_host) return fail(HH_ERR_INVALID_ARG, "particle pointer is NULL");
    if (!rgb8_host) return fail(HH_ERR_INVALID_ARG, "image pointer array is NULL");
    for (size_t v = 0; v < p->cams.size(); ++v)
        if (!rgb8_host[v]) return fail(HH_ERR_INVALID_ARG, "view %zu: image pointer is NULL", v);
    const uint64_t f = p->next_frame;
    PipeSlot& s = p->slot[f % kSlots];
    const DeviceScope on(p->device);
    if (s.frame >= 0) {  // the slot's previous frame must be done with its buffers
        const cudaError_t q = wait_event(s.downloaded, kSubmitWaitMs);
        if (q == cudaErrorNotReady)
            return fail(HH_ERR_TIMEOUT, "frame %lld still running after %d ms",
                        static_cast<long long>(s.frame), kSubmitWaitMs);
        if (q != cudaSuccess) return hh::cuda_fail(q, "previous frame");
    }
    cudaError_t e = cudaSuccess;
    if (n > 0)
        e = cudaMemcpyAsync(s.parts_dev, xyzm_host, static_cast<size_t>(n) * 16,
                            cudaMemcpyHostToDevice, p->up);
    if (e == cudaSuccess) e = cudaEventRecord(s.uploaded, p->up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s.build, s.uploaded, 0);
    if (e != cudaSuccess) return hh::cuda_fail(e, "particle upload");
    // the slot's previous march (frame t-2) is done: its images were downloaded
    const hh_particles parts{s.parts_dev, n};
    hh_status st = hh_volume_rebuild(s.vol, &parts, p->K, s.build);
    if (st != HH_OK) return st;
    e = cudaEventRecord(s.built, s.build);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s.march, s.built, 0);
    if (e != cudaSuccess) return hh::cuda_fail(e, "volume build");
    if (p->batched)
        st = hh_batch_launch_graph(s.batch, s.march);
    else
        st = hh_trace(s.vol, p->cams.data(), static_cast<int>(p->cams.size()), &p->params,
                      &p->bg, s.outs.data(), s.march);
    if (st != HH_OK) return st;
    e = cudaEventRecord(s.rendered, s.march);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->down, s.rendered, 0);
    for (size_t v = 0; v < p->cams.size() && e == cudaSuccess; ++v)
        e = cudaMemcpyAsync(rgb8_host[v], s.outs[v].rgb8, p->view_bytes[v],
                            cudaMemcpyDeviceToHost, p->down);
    if (e == cudaSuccess) e = cudaEventRecord(s.downloaded, p->down);
    if (e != cudaSuccess) return hh::cuda_fail(e, "image download");
    s.frame = static_cast<int64_t>(f);
    p->next_frame = f + 1;
    if (frame) *frame = f;
    return hh::ok();
}

hh_status hh_pipeline_wait(hh_pipeline p, uint64_t frame, int timeout_ms) {
    using hh::fail;
    if (!p) return fail(HH_ERR_INVALID_ARG, "pipeline is NULL");
    if (frame >= p->next_frame)
        return fail(HH_ERR_NOT_FOUND, "frame %llu has not been submitted",
                    static_cast<unsigned long long>(frame));
    const PipeSlot& s = p->slot[frame % kSlots];
    if (s.frame != static_cast<int64_t>(frame)) return hh::ok();  // the slot moved on: done
    const DeviceScope on(p->device);
    const cudaError_t q = wait_event(s.downloaded, timeout_ms < 0 ? 0 : timeout_ms);
    if (q == cudaErrorNotReady)
        return fail(HH_ERR_TIMEOUT, "frame %llu not done after %d ms",
                    static_cast<unsigned long long>(frame), timeout_ms);
    if (q != cudaSuccess) return hh::cuda_fail(q, "frame");
    return hh::ok();
}

hh_status hh_pipeline_volume(hh_pipeline p, hh_volume* vol) {
    if (!p || !vol) return hh::fail(HH_ERR_INVALID_ARG, "pipeline or output is NULL");
    // the slot of the last submitted frame (slot 0 before any)
    *vol = p->slot[p->next_frame == 0 ? 0 : (p->next_frame - 1) % kSlots].vol;
    return hh::ok();
}

hh_status hh_pipeline_free(hh_pipeline p) {
    if (!p) return hh::ok();
    const DeviceScope on(p->device);
    cudaError_t e = cudaSuccess;
    for (const PipeSlot& s : p->slot) {
        if (s.frame < 0) continue;
        const cudaError_t q = wait_event(s.downloaded, kSubmitWaitMs);
        if (q == cudaErrorNotReady)  // its buffers are still in use: keep them
            return hh::fail(HH_ERR_TIMEOUT, "frame %lld still running after %d ms",
                            static_cast<long long>(s.frame), kSubmitWaitMs);
        if (e == cudaSuccess) e = q;
    }
    delete p;
    if (e != cudaSuccess) return hh::cuda_fail(e, "pipeline frames");
    return hh::ok();
}

}  // extern "C"
