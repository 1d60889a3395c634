// Render server with continuous batching (hh_serve_*).
//
// Requests (1..256 views of one simulation frame's volume) are admitted as
// soon as a slot is free and their output buffers fit in the server's
// device-memory budget; each admitted request runs as one persistent batched
// launch (the hh_batch kernel) on its slot's stream, so requests that arrive
// while others are on the GPU overlap with them on the device. A worker
// thread watches the slots' completion events and admits waiting requests as
// slots and memory free up. Requests that do not fit wait (others may pass
// them); a request larger than the whole budget is refused at submission.
// All waits on the host are bounded.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "hh_internal.h"
#include "pool.h"

namespace {

constexpr int kMaxViews = 256;
constexpr int kMaxSlots = 64;

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

enum State { PENDING, RUNNING, DONE, CANCELLED, FAILED };

struct Request {
    uint64_t ticket = 0;
    int64_t frame = 0;
    std::vector<hh_camera> cams;
    hh_step_params params{};
    hh_background bg{};
    int outputs = HH_OUT_RGB;
    size_t bytes = 0;     // output bytes in the pool
    size_t offset = 0;    // pool offset once admitted
    std::vector<hh_view_out> outs;
    State state = PENDING;
    bool cancel_requested = false;
    int slot = -1;
    hh_status error = HH_OK;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void* table_host = nullptr;  // pinned staging for the view table
    void* table_dev = nullptr;
    unsigned* counter = nullptr;
    uint64_t ticket = 0;         // 0 when free
};

// Output bytes of one view for the requested outputs.
size_t view_bytes(const hh_camera& c, int outputs) {
    const size_t px = static_cast<size_t>(c.width) * c.height;
    size_t b = 0;
    if (outputs & HH_OUT_RGB) b += align256(px * 12);
    if (outputs & HH_OUT_RGB8) b += align256(px * 3);
    if (outputs & HH_OUT_EXIT) b += 2 * align256(px * 12);
    if (outputs & HH_OUT_STEPS) b += 2 * align256(px * 4);
    return b;
}

}  // namespace

struct hh_server_s {
    int device = 0;
    int sm_count = 0;
    hh_batch_config cfg{128, 0, 32, 8};
    char* pool_base = nullptr;
    hh::OffsetPool pool;
    std::vector<Slot> slots;
    std::map<int64_t, hh_volume> frames;
    std::map<int64_t, int> frame_users;  // running requests per frame
    std::map<uint64_t, Request> reqs;
    std::deque<uint64_t> pending;
    std::mutex mu;
    std::condition_variable cv;  // signalled on completions and state changes
    std::condition_variable work;  // wakes the worker
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    hh_serve_stats stats{};
    double max_bypass_ms = 200.0;  // a waiting request older than this blocks others

    void run();
    void complete_slots();
    void admit();
    hh_status launch(Request& r, int slot);
};

hh_status hh_server_s::launch(Request& r, int si) {
    Slot& s = slots[si];
    // carve this request's outputs out of its pool block
    char* p = pool_base + r.offset;
    r.outs.resize(r.cams.size());
    for (size_t v = 0; v < r.cams.size(); ++v) {
        const size_t px = static_cast<size_t>(r.cams[v].width) * r.cams[v].height;
        hh_view_out& o = r.outs[v];
        o = hh_view_out{};
        if (r.outputs & HH_OUT_RGB) {
            o.rgb = reinterpret_cast<float*>(p);
            p += align256(px * 12);
        }
        if (r.outputs & HH_OUT_RGB8) {
            o.rgb8 = reinterpret_cast<uint8_t*>(p);
            p += align256(px * 3);
        }
        if (r.outputs & HH_OUT_EXIT) {
            o.exit_pos = reinterpret_cast<float*>(p);
            p += align256(px * 12);
            o.exit_dir = reinterpret_cast<float*>(p);
            p += align256(px * 12);
        }
        if (r.outputs & HH_OUT_STEPS) {
            o.steps = reinterpret_cast<int32_t*>(p);
            p += align256(px * 4);
            o.flags = reinterpret_cast<uint32_t*>(p);
            p += align256(px * 4);
        }
    }
    const int n = static_cast<int>(r.cams.size());
    const int tiles = hh::build_view_table(r.cams.data(), r.outs.data(), n, cfg.tile_w,
                                           s.table_host);
    if (tiles < 0) return hh::fail(HH_ERR_INVALID_ARG, "request has too many pixels");
    cudaError_t e = cudaMemcpyAsync(s.table_dev, s.table_host, n * hh::view_record_bytes(),
                                    cudaMemcpyHostToDevice, s.stream);
    if (e == cudaSuccess)
        e = hh::launch_batch(frames[r.frame], r.params, r.bg, s.table_dev, n, tiles, s.counter, cfg,
                             sm_count, s.stream);
    if (e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
    if (e != cudaSuccess) return hh::cuda_fail(e, "request launch");
    return HH_OK;
}

void hh_server_s::complete_slots() {
    for (size_t i = 0; i < slots.size(); ++i) {
        Slot& s = slots[i];
        if (!s.ticket) continue;
        const cudaError_t q = cudaEventQuery(s.done);
        if (q == cudaErrorNotReady) continue;
        auto it = reqs.find(s.ticket);
        if (it != reqs.end()) {
            Request& r = it->second;
            r.t_done = now_ms();
            if (q != cudaSuccess) {
                r.state = FAILED;
                r.error = HH_ERR_CUDA;
                ++stats.failed;
            } else if (r.cancel_requested) {
                r.state = CANCELLED;
                ++stats.cancelled;
            } else {
                r.state = DONE;
                ++stats.completed;
                for (const auto& c : r.cams)
                    stats.rays_completed += static_cast<uint64_t>(c.width) * c.height;
            }
            if (--frame_users[r.frame] == 0) frame_users.erase(r.frame);
            if (r.state == CANCELLED) {  // nobody will read it: give the memory back
                pool.release(r.offset);
            }
        } else {
            cudaGetLastError();
        }
        s.ticket = 0;
        --stats.running;
        cv.notify_all();
    }
}

void hh_server_s::admit() {
    const double t = now_ms();
    for (auto it = pending.begin(); it != pending.end();) {
        auto rit = reqs.find(*it);
        if (rit == reqs.end()) {  // released or cancelled while waiting
            it = pending.erase(it);
            continue;
        }
        Request& r = rit->second;
        int free_slot = -1;
        for (size_t i = 0; i < slots.size(); ++i)
            if (!slots[i].ticket) {
                free_slot = static_cast<int>(i);
                break;
            }
        if (free_slot < 0) return;
        if (!frames.count(r.frame)) {  // its volume has not arrived yet
            ++it;
            continue;
        }
        size_t off = 0;
        if (!pool.alloc(r.bytes, &off)) {
            // not enough memory now; later (smaller) requests may pass it
            // unless it has already waited too long
            if (t - r.t_submit > max_bypass_ms) return;
            ++it;
            continue;
        }
        r.offset = off;
        hh_status st = launch(r, free_slot);
        if (st != HH_OK) {
            pool.release(off);
            r.state = FAILED;
            r.error = st;
            ++stats.failed;
            --stats.pending;
            it = pending.erase(it);
            cv.notify_all();
            continue;
        }
        r.state = RUNNING;
        r.slot = free_slot;
        r.t_admit = t;
        slots[free_slot].ticket = r.ticket;
        ++frame_users[r.frame];
        ++stats.admitted;
        ++stats.running;
        --stats.pending;
        it = pending.erase(it);
    }
}

void hh_server_s::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    while (!stop) {
        complete_slots();
        admit();
        const bool busy = stats.running > 0;
        // poll completions every 20 us while work is on the GPU; otherwise
        // sleep until a submission or state change (re-checking every 5 ms)
        work.wait_for(lock, busy ? std::chrono::microseconds(20) : std::chrono::milliseconds(5));
    }
}

extern "C" {

hh_status hh_serve_create(size_t mem_budget_bytes, int max_slots, hh_server* out) {
    if (!out) return hh::fail(HH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_slots > kMaxSlots)
        return hh::fail(HH_ERR_INVALID_ARG, "max_slots must be in [1, %d]", kMaxSlots);
    if (mem_budget_bytes < 4096) return hh::fail(HH_ERR_INVALID_ARG, "budget below 4 KiB");
    hh_server S = new (std::nothrow) hh_server_s();
    if (!S) return hh::fail(HH_ERR_OOM, "host allocation failed");
    cudaGetDevice(&S->device);
    cudaDeviceGetAttribute(&S->sm_count, cudaDevAttrMultiProcessorCount, S->device);
    cudaError_t e = hh::dev_alloc(reinterpret_cast<void**>(&S->pool_base), mem_budget_bytes);
    if (e != cudaSuccess) {
        delete S;
        return hh::cuda_fail(e, "server memory budget");
    }
    S->pool.reset(mem_budget_bytes, 256);
    S->slots.resize(max_slots);
    for (auto& s : S->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = hh::host_alloc(&s.table_host, kMaxViews * hh::view_record_bytes());
        if (e == cudaSuccess) e = hh::dev_alloc(&s.table_dev, kMaxViews * hh::view_record_bytes());
        if (e == cudaSuccess) e = hh::dev_alloc(reinterpret_cast<void**>(&s.counter), sizeof(unsigned));
    }
    if (e != cudaSuccess) {
        hh_status st = hh::cuda_fail(e, "server slots");
        hh_serve_destroy(S);
        return st;
    }
    S->stats.pool_capacity = S->pool.capacity();
    S->worker = std::thread([S] { S->run(); });
    *out = S;
    return hh::ok();
}

hh_status hh_serve_set_config(hh_server S, const hh_batch_config* cfg) {
    if (!S || !cfg) return hh::fail(HH_ERR_INVALID_ARG, "server or config is NULL");
    if (cfg->block_threads < 32 || cfg->block_threads > 256 || cfg->block_threads % 32 ||
        cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 64 || cfg->refill_min < 1 ||
        cfg->refill_min > 32 || (cfg->tile_w != 4 && cfg->tile_w != 8 && cfg->tile_w != 16))
        return hh::fail(HH_ERR_INVALID_ARG, "invalid launch configuration");
    std::lock_guard<std::mutex> lock(S->mu);
    S->cfg = *cfg;
    return hh::ok();
}

hh_status hh_serve_put_volume(hh_server S, int64_t frame_id, hh_volume vol) {
    if (!S || !vol) return hh::fail(HH_ERR_INVALID_ARG, "server or volume is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->frame_users.count(frame_id))
        return hh::fail(HH_ERR_BUSY, "frame %lld is being rendered", static_cast<long long>(frame_id));
    S->frames[frame_id] = vol;
    S->work.notify_one();
    return hh::ok();
}

hh_status hh_serve_remove_volume(hh_server S, int64_t frame_id) {
    if (!S) return hh::fail(HH_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    if (!S->frames.count(frame_id))
        return hh::fail(HH_ERR_NOT_FOUND, "no frame %lld", static_cast<long long>(frame_id));
    if (S->frame_users.count(frame_id))
        return hh::fail(HH_ERR_BUSY, "frame %lld is being rendered", static_cast<long long>(frame_id));
    S->frames.erase(frame_id);
    return hh::ok();
}

hh_status hh_serve_submit(hh_server S, int64_t frame_id, const hh_camera* cams, int n_views,
                          const hh_step_params* params, const hh_background* bg, int outputs,
                          uint64_t* ticket) {
    if (!S || !ticket) return hh::fail(HH_ERR_INVALID_ARG, "server or ticket is NULL");
    if (n_views < 1 || n_views > kMaxViews || !cams)
        return hh::fail(HH_ERR_INVALID_ARG, "a request has 1 to %d views", kMaxViews);
    if (outputs & ~(HH_OUT_RGB | HH_OUT_EXIT | HH_OUT_STEPS | HH_OUT_RGB8))
        return hh::fail(HH_ERR_INVALID_ARG, "unknown output bits");
    if (!(outputs & (HH_OUT_RGB | HH_OUT_RGB8))) outputs |= HH_OUT_RGB;  // an image is always made
    hh_status st = hh::check_params(params);
    if (st != HH_OK) return st;
    if ((st = hh::check_background(bg)) != HH_OK) return st;
    Request r;
    for (int i = 0; i < n_views; ++i) {
        if ((st = hh::check_camera(cams[i], i)) != HH_OK) return st;
        r.bytes += view_bytes(cams[i], outputs);
    }
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->pool.footprint(r.bytes) > S->pool.capacity()) {
        ++S->stats.rejected;
        return hh::fail(HH_ERR_OOM, "request needs %zu bytes of outputs; the budget is %zu",
                        r.bytes, S->pool.capacity());
    }
    r.ticket = S->next_ticket++;
    r.frame = frame_id;
    r.cams.assign(cams, cams + n_views);
    r.params = *params;
    r.bg = *bg;
    r.outputs = outputs;
    r.t_submit = now_ms();
    *ticket = r.ticket;
    S->pending.push_back(r.ticket);
    S->reqs.emplace(r.ticket, std::move(r));
    ++S->stats.submitted;
    ++S->stats.pending;
    S->work.notify_one();
    return hh::ok();
}

static hh_status status_of(const Request& r, double* latency_ms) {
    switch (r.state) {
        case DONE:
            if (latency_ms) *latency_ms = r.t_done - r.t_submit;
            return HH_OK;
        case CANCELLED:
            return hh::fail(HH_ERR_CANCELLED, "request %llu was cancelled",
                            static_cast<unsigned long long>(r.ticket));
        case FAILED:
            return hh::fail(r.error == HH_OK ? HH_ERR_CUDA : r.error, "request %llu failed",
                            static_cast<unsigned long long>(r.ticket));
        default:
            return HH_ERR_BUSY;
    }
}

hh_status hh_serve_poll(hh_server S, uint64_t ticket, double* latency_ms) {
    if (!S) return hh::fail(HH_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end())
        return hh::fail(HH_ERR_NOT_FOUND, "no request %llu", static_cast<unsigned long long>(ticket));
    return status_of(it->second, latency_ms);
}

hh_status hh_serve_wait(hh_server S, uint64_t ticket, int timeout_ms, double* latency_ms) {
    if (!S) return hh::fail(HH_ERR_INVALID_ARG, "server is NULL");
    if (timeout_ms < 0) return hh::fail(HH_ERR_INVALID_ARG, "timeout must be >= 0");
    std::unique_lock<std::mutex> lock(S->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end())
            return hh::fail(HH_ERR_NOT_FOUND, "no request %llu",
                            static_cast<unsigned long long>(ticket));
        const State st = it->second.state;
        if (st != PENDING && st != RUNNING) return status_of(it->second, latency_ms);
        if (S->cv.wait_until(lock, deadline) == std::cv_status::timeout) {
            it = S->reqs.find(ticket);
            if (it != S->reqs.end() && it->second.state != PENDING && it->second.state != RUNNING)
                return status_of(it->second, latency_ms);
            return hh::fail(HH_ERR_TIMEOUT, "request %llu not done after %d ms",
                            static_cast<unsigned long long>(ticket), timeout_ms);
        }
    }
}

hh_status hh_serve_view(hh_server S, uint64_t ticket, int view, hh_view_out* out) {
    if (!S || !out) return hh::fail(HH_ERR_INVALID_ARG, "server or out is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end())
        return hh::fail(HH_ERR_NOT_FOUND, "no request %llu", static_cast<unsigned long long>(ticket));
    const Request& r = it->second;
    if (r.state != DONE) return status_of(r, nullptr);
    if (view < 0 || view >= static_cast<int>(r.outs.size()))
        return hh::fail(HH_ERR_INVALID_ARG, "view %d out of range", view);
    *out = r.outs[view];
    return hh::ok();
}

hh_status hh_serve_release(hh_server S, uint64_t ticket) {
    if (!S) return hh::fail(HH_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end())
        return hh::fail(HH_ERR_NOT_FOUND, "no request %llu", static_cast<unsigned long long>(ticket));
    Request& r = it->second;
    if (r.state == RUNNING || (r.state == PENDING))
        return hh::fail(HH_ERR_BUSY, "request %llu is not finished (cancel it first)",
                        static_cast<unsigned long long>(ticket));
    // a finished request still holds its outputs (a cancelled one gave them
    // back when its launch ended; one that failed to launch never had any)
    if ((r.state == DONE || r.state == FAILED) && r.slot >= 0) S->pool.release(r.offset);
    S->reqs.erase(it);
    S->work.notify_one();
    return hh::ok();
}

hh_status hh_serve_cancel(hh_server S, uint64_t ticket) {
    if (!S) return hh::fail(HH_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end())
        return hh::fail(HH_ERR_NOT_FOUND, "no request %llu", static_cast<unsigned long long>(ticket));
    Request& r = it->second;
    if (r.state == PENDING) {
        r.state = CANCELLED;
        r.t_done = now_ms();
        S->pending.erase(std::remove(S->pending.begin(), S->pending.end(), ticket),
                         S->pending.end());
        --S->stats.pending;
        ++S->stats.cancelled;
        S->cv.notify_all();
    } else if (r.state == RUNNING) {
        r.cancel_requested = true;  // its launch finishes; the result is discarded
    }
    return hh::ok();
}

hh_status hh_serve_get_stats(hh_server S, hh_serve_stats* out) {
    if (!S || !out) return hh::fail(HH_ERR_INVALID_ARG, "server or out is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    *out = S->stats;
    out->pool_used = S->pool.used();
    out->pool_capacity = S->pool.capacity();
    return hh::ok();
}

hh_status hh_serve_destroy(hh_server S) {
    if (!S) return hh::ok();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
        S->work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (auto& s : S->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.done) cudaEventDestroy(s.done);
        if (s.table_host) hh::host_free(s.table_host);
        if (s.table_dev) hh::dev_free(s.table_dev);
        if (s.counter) hh::dev_free(s.counter);
    }
    hh::dev_free(S->pool_base);
    delete S;
    return hh::ok();
}

}  // extern "C"
