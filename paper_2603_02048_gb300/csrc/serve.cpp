// Render server with ray-level continuous batching (hh_serve_*).
//
// One persistent worker kernel serves every request: the host publishes each
// admitted request ("job": its volume, its view records and its tile count)
// into a device queue while the worker runs, and the worker's warps take
// 32-pixel tiles of the oldest job that still has some, so a new request's
// rays start as soon as warps free up, alongside the rays of the requests
// already on the GPU. The warp that finishes a job's last tile raises the
// job's flag in host-mapped memory; a host thread watches the flags, admits
// waiting requests as in-flight capacity and output memory free up, and
// launches the worker again whenever published work finds it gone (its warps
// leave after a short idle spell). Publication uses copies only (the copy
// engine runs beside the persistent kernel): the job's view records, then its
// entry, then the published-job count, in order on one control stream.
//
// Requests share the worker's launch-wide arguments (grid dimensions,
// storage, step schedule, background): a request of another schedule or
// scene waits until the running ones are done, then the worker restarts with
// its arguments. Waiting requests are admitted smallest first (fewest rays),
// except that a request waiting over kAgeMs goes ahead of all younger ones.
// A request whose outputs exceed the whole budget is refused; requests that
// do not fit yet wait (others may pass them unless they have waited over
// 200 ms); requests for a frame not yet put wait for it. All
// host waits are bounded, and so is every wait of the worker.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "admission.h"
#include "hh_internal.h"
#include "pool.h"

namespace {

constexpr int kMaxViews = 256;         // views per request
constexpr int kMaxSlots = 64;          // requests on the GPU at once
constexpr int kJobs = 1 << 14;         // job entries between queue resets
constexpr int kViewRecords = 1 << 16;  // view records between queue resets
constexpr double kAgeMs = 50.0;  // admission: a request waiting this long goes first
constexpr unsigned long long kIdleNs = 2000000;   // a worker warp leaves after 2 ms without work
constexpr unsigned long long kEntryNs = 5000000;  // a published entry missing for 5 ms fails its job

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
    size_t bytes = 0;   // output bytes in the pool
    uint64_t rays = 0;  // primary rays of all its views
    size_t offset = 0;  // pool offset once admitted
    bool has_memory = false;
    std::vector<hh_view_out> outs;
    State state = PENDING;
    bool cancel_requested = false;
    int job = -1;  // its job number while published
    hh_status error = HH_OK;
    double t_submit = 0, t_admit = 0, t_done = 0;
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

bool same_plane(const hh_plane& a, const hh_plane& b) {
    for (int i = 0; i < 3; ++i)
        if (a.origin[i] != b.origin[i] || a.u[i] != b.u[i] || a.v[i] != b.v[i]) return false;
    return a.rgb8_dev == b.rgb8_dev && a.width == b.width && a.height == b.height;
}

// Whether request `a` on volume `va` can join a worker launched with schedule
// `p`, background `g` and grid `vb` (its launch-wide arguments).
bool same_class(const Request& a, const hh_volume_s* va, const hh_step_params& p,
                const hh_background& g, const hh_volume_s* vb) {
    if (va->nx != vb->nx || va->ny != vb->ny || va->nz != vb->nz || va->storage != vb->storage)
        return false;
    const hh_step_params& q = a.params;
    if (p.stepper != q.stepper || p.adaptive != q.adaptive || p.h_fixed != q.h_fixed ||
        p.h_min != q.h_min || p.h_max != q.h_max || p.theta_max != q.theta_max ||
        p.eps != q.eps || p.max_steps != q.max_steps)
        return false;
    const hh_background& h = a.bg;
    if (g.rgb8_dev != h.rgb8_dev || g.width != h.width || g.height != h.height ||
        g.n_planes != h.n_planes)
        return false;
    for (int k = 0; k < g.n_planes && k < HH_MAX_PLANES; ++k)
        if (!same_plane(g.planes[k], h.planes[k])) return false;
    return true;
}

}  // namespace

struct hh_server_s {
    int device = 0;
    int sm_count = 0;
    int max_inflight = 1;
    hh_batch_config cfg{128, 0, 32, 8, 0, 0};
    char* pool_base = nullptr;
    hh::OffsetPool pool;
    // the queue on the device
    hh::ServeJob* jobs_dev = nullptr;
    char* views_dev = nullptr;
    unsigned* claimed_dev = nullptr;
    unsigned* done_dev = nullptr;
    int* ctl_dev = nullptr;  // [0] jobs published, [1] first open job, [2] stop request,
                             // [3] idle warps, [4] leave flag and [5] started warps of
                             // the running launch
    // pinned staging of what the control stream copies
    hh::ServeJob* jobs_host = nullptr;
    char* views_host = nullptr;
    int* pub_host = nullptr;  // slot j holds j + 1: the count that publishes job j
    int* consts_host = nullptr;  // {0, 1}: sources of the stop request's copies
    // host-mapped flags (host pointers; the worker gets their device aliases)
    unsigned* flags_host = nullptr;
    int* hctl_host = nullptr;  // [1] exit reason of the last worker launch
    unsigned* flags_alias = nullptr;
    int* hctl_alias = nullptr;
    cudaStream_t ctl_stream = nullptr, work_stream = nullptr;
    cudaEvent_t published = nullptr, worker_done = nullptr, reset_done = nullptr;
    bool worker_running = false;
    bool stop_requested = false;  // the device stop flag is set
    int next_job = 0, next_view = 0;
    std::vector<uint64_t> job_ticket;  // per job number: its request's ticket (0: none)
    std::vector<int> inflight;         // job numbers published and not yet finished
    std::vector<size_t> quarantine;    // pool blocks of failed jobs, freed once no worker runs
    uint64_t published_total = 0;      // jobs published since creation
    // the worker's launch-wide arguments (valid while have_class)
    bool have_class = false;
    hh_step_params cls_params{};
    hh_background cls_bg{};
    hh_volume cls_vol = nullptr;
    std::map<int64_t, hh_volume> frames;
    std::map<int64_t, int> frame_users;  // published requests per frame
    std::map<uint64_t, Request> reqs;
    std::deque<uint64_t> pending;
    std::mutex mu;
    std::condition_variable cv;    // signalled on completions and state changes
    std::condition_variable work;  // wakes the host thread
    std::thread host_thread;
    bool stop = false;
    uint64_t next_ticket = 1;
    hh_serve_stats stats{};
    double max_bypass_ms = 200.0;  // a waiting request older than this blocks others

    void run();
    void complete_jobs();
    void check_worker();
    void fail_inflight(hh_status err);
    void admit();
    void launch_worker();
    void reset_queue();
    void request_stop();
    hh_status publish(Request& r);
    void finish(Request& r, State st, hh_status err);
};

// Marks a published request finished and returns what it no longer needs.
void hh_server_s::finish(Request& r, State st, hh_status err) {
    r.t_done = now_ms();
    r.state = st;
    r.error = err;
    if (st == DONE) {
        ++stats.completed;
        for (const auto& c : r.cams)
            stats.rays_completed += static_cast<uint64_t>(c.width) * c.height;
    } else if (st == CANCELLED) {
        ++stats.cancelled;
    } else {
        ++stats.failed;
    }
    if (--frame_users[r.frame] == 0) frame_users.erase(r.frame);
    if (st == CANCELLED && r.has_memory) {  // nobody will read it
        pool.release(r.offset);
        r.has_memory = false;
    }
    if (st == FAILED && r.has_memory) {  // a warp may still write it: freed once no worker runs
        quarantine.push_back(r.offset);
        r.has_memory = false;
    }
    --stats.running;
    cv.notify_all();
}

hh_status hh_server_s::publish(Request& r) {
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
    const size_t rec = hh::view_record_bytes();
    const int j = next_job;
    char* stage = views_host + static_cast<size_t>(next_view) * rec;
    const int tiles = hh::build_view_table(r.cams.data(), r.outs.data(), n, cfg.tile_w, stage);
    if (tiles < 0) return hh::fail(HH_ERR_INVALID_ARG, "request has too many pixels");
    const hh_volume vol = frames[r.frame];
    hh::ServeJob& e = jobs_host[j];
    e.vol = vol->data;
    e.scales = vol->scales_dev;
    e.view_begin = next_view;
    e.n_views = n;
    e.n_tiles = tiles;
    e.seq = j;
    pub_host[j] = j + 1;
    // test hook: HH_SERVE_DROP_ENTRY=k leaves out the entry copy of the k-th
    // job published since the server's creation (its count is still
    // published), so the worker's bounded wait for the entry runs out
    ++published_total;
    const char* drop = std::getenv("HH_SERVE_DROP_ENTRY");
    const bool skip_entry = drop && *drop && std::strtoull(drop, nullptr, 10) == published_total;
    cudaError_t err = cudaMemcpyAsync(views_dev + static_cast<size_t>(next_view) * rec, stage,
                                      n * rec, cudaMemcpyHostToDevice, ctl_stream);
    if (err == cudaSuccess && !skip_entry)
        err = cudaMemcpyAsync(jobs_dev + j, jobs_host + j, sizeof(hh::ServeJob),
                              cudaMemcpyHostToDevice, ctl_stream);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(ctl_dev, pub_host + j, sizeof(int), cudaMemcpyHostToDevice,
                              ctl_stream);
    if (err == cudaSuccess) err = cudaEventRecord(published, ctl_stream);
    if (err != cudaSuccess) return hh::cuda_fail(err, "publishing a request");
    job_ticket[j] = r.ticket;
    r.job = j;
    ++next_job;
    next_view += n;
    inflight.push_back(j);
    return HH_OK;
}

void hh_server_s::complete_jobs() {
    for (size_t i = 0; i < inflight.size();) {
        const int j = inflight[i];
        const unsigned f = reinterpret_cast<volatile unsigned*>(flags_host)[j];
        if (f == 0) {
            ++i;
            continue;
        }
        inflight[i] = inflight.back();
        inflight.pop_back();
        auto it = reqs.find(job_ticket[j]);
        job_ticket[j] = 0;
        if (it == reqs.end()) continue;
        Request& r = it->second;
        if (f == hh::HH_JOB_FAILED) {
            ++stats.entry_timeouts;
            finish(r, FAILED, HH_ERR_TIMEOUT);
        } else {
            finish(r, r.cancel_requested ? CANCELLED : DONE, HH_OK);
        }
    }
}

void hh_server_s::fail_inflight(hh_status err) {
    for (int j : inflight) {
        auto it = reqs.find(job_ticket[j]);
        job_ticket[j] = 0;
        if (it != reqs.end()) finish(it->second, FAILED, err);
    }
    inflight.clear();
}

void hh_server_s::check_worker() {
    if (!worker_running) return;
    const cudaError_t q = cudaEventQuery(worker_done);
    if (q == cudaErrorNotReady) return;
    worker_running = false;
    if (q != cudaSuccess) {  // the launch failed: fail what it held
        cudaGetLastError();
        fail_inflight(HH_ERR_CUDA);
        return;
    }
    if (reinterpret_cast<volatile int*>(hctl_host)[1] != hh::HH_WORKER_STOPPED)
        ++stats.worker_idle_exits;
    complete_jobs();  // flags raised just before the worker left
    for (size_t off : quarantine) pool.release(off);
    quarantine.clear();
    cv.notify_all();
}

// Sets the device stop flag (a copy: it reaches a running worker).
void hh_server_s::request_stop() {
    if (stop_requested) return;
    if (cudaMemcpyAsync(ctl_dev + 2, consts_host + 1, sizeof(int), cudaMemcpyHostToDevice,
                        ctl_stream) == cudaSuccess)
        stop_requested = true;
    else
        cudaGetLastError();
}

void hh_server_s::launch_worker() {
    hctl_host[1] = 0;
    cudaError_t e = cudaSuccess;
    if (stop_requested) {  // cleared before the launch, which waits for `published`
        e = cudaMemcpyAsync(ctl_dev + 2, consts_host, sizeof(int), cudaMemcpyHostToDevice,
                            ctl_stream);
        if (e == cudaSuccess) e = cudaEventRecord(published, ctl_stream);
        stop_requested = false;
    }
    hh::ServeWorkerArgs W;
    W.jobs = jobs_dev;
    W.views = views_dev;
    W.claimed = claimed_dev;
    W.done = done_dev;
    W.n_jobs = ctl_dev;
    W.first_open = ctl_dev + 1;
    W.stop = ctl_dev + 2;
    W.idle_warps = ctl_dev + 3;
    W.leave = ctl_dev + 4;
    W.started_warps = ctl_dev + 5;
    W.host_done = flags_alias;
    W.host_ctl = hctl_alias;
    W.tile_w = cfg.tile_w;
    W.idle_ns = kIdleNs;
    W.entry_ns = kEntryNs;
    const int bps = cfg.blocks_per_sm > 0
                        ? cfg.blocks_per_sm
                        : hh::serve_worker_blocks_per_sm(cls_vol->storage, cls_params.stepper,
                                                         cls_params.adaptive, cfg.block_threads);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(work_stream, published, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl_dev + 3, 0, 3 * sizeof(int), work_stream);
    if (e == cudaSuccess)
        e = hh::launch_serve_worker(cls_vol, cls_params, cls_bg, W, sm_count * bps,
                                    cfg.block_threads, work_stream);
    if (e == cudaSuccess) e = cudaEventRecord(worker_done, work_stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail_inflight(HH_ERR_CUDA);
        return;
    }
    worker_running = true;
    ++stats.worker_launches;
}

// Clears the queue back to job number 0 (only while no worker runs and
// nothing is in flight): the counters and the entries' numbers on the
// device, the flags on the host. Later publications wait for it.
void hh_server_s::reset_queue() {
    cudaError_t e = cudaMemsetAsync(claimed_dev, 0, next_job * sizeof(unsigned), work_stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(done_dev, 0, next_job * sizeof(unsigned), work_stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(jobs_dev, 0xff, next_job * sizeof(hh::ServeJob), work_stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl_dev, 0, 6 * sizeof(int), work_stream);
    if (e == cudaSuccess) e = cudaEventRecord(reset_done, work_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctl_stream, reset_done, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return;  // numbering goes on; the queue limits stop admission until a reset works
    }
    std::memset(flags_host, 0, next_job * sizeof(unsigned));
    stop_requested = false;
    next_job = 0;
    next_view = 0;
}

void hh_server_s::admit() {
    const double t = now_ms();
    // smallest request first, except that a request waiting longer than
    // kAgeMs goes ahead of every younger one (oldest first among them);
    // tickets no longer known (released or cancelled) go last
    std::stable_sort(pending.begin(), pending.end(), [&](uint64_t a, uint64_t b) {
        auto ia = reqs.find(a), ib = reqs.find(b);
        if (ia == reqs.end() || ib == reqs.end()) return ia != reqs.end() && ib == reqs.end();
        return hh::admit_before({ia->second.t_submit, ia->second.rays},
                                {ib->second.t_submit, ib->second.rays}, t, kAgeMs);
    });
    for (auto it = pending.begin(); it != pending.end();) {
        auto rit = reqs.find(*it);
        if (rit == reqs.end()) {  // released or cancelled while waiting
            it = pending.erase(it);
            continue;
        }
        Request& r = rit->second;
        if (static_cast<int>(inflight.size()) >= max_inflight) return;
        auto fit = frames.find(r.frame);
        if (fit == frames.end()) {  // its volume has not arrived yet
            ++it;
            continue;
        }
        if (!have_class || !same_class(r, fit->second, cls_params, cls_bg, cls_vol)) {
            if (!inflight.empty() || worker_running) {
                // another schedule or scene runs: this one waits for it to
                // drain (an idle worker is told to stop)
                if (inflight.empty()) request_stop();
                if (t - r.t_submit > max_bypass_ms) return;
                ++it;
                continue;
            }
            have_class = true;
            cls_params = r.params;
            cls_bg = r.bg;
            cls_vol = fit->second;
        }
        if (next_job >= kJobs || next_view + static_cast<int>(r.cams.size()) > kViewRecords)
            return;  // the queue is full until it drains and resets
        size_t off = 0;
        if (!pool.alloc(r.bytes, &off)) {
            // not enough memory now; later (smaller) requests may pass it
            // unless it has already waited too long
            if (t - r.t_submit > max_bypass_ms) return;
            ++it;
            continue;
        }
        r.offset = off;
        r.has_memory = true;
        hh_status st = publish(r);
        if (st != HH_OK) {
            pool.release(off);
            r.has_memory = false;
            r.state = FAILED;
            r.error = st;
            ++stats.failed;
            --stats.pending;
            it = pending.erase(it);
            cv.notify_all();
            continue;
        }
        r.state = RUNNING;
        r.t_admit = t;
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
        complete_jobs();
        check_worker();
        if (inflight.empty() && !worker_running) {
            if (next_job > 0) reset_queue();
            have_class = false;
        }
        admit();
        if (!inflight.empty() && !worker_running) launch_worker();
        const bool busy = !inflight.empty() || worker_running;
        // poll the flags every 20 us while work is on the GPU; otherwise
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
    S->max_inflight = max_slots;
    S->job_ticket.assign(kJobs, 0);
    const size_t rec = hh::view_record_bytes();
    cudaError_t e = hh::dev_alloc(reinterpret_cast<void**>(&S->pool_base), mem_budget_bytes);
    if (e != cudaSuccess) {
        delete S;
        return hh::cuda_fail(e, "server memory budget");
    }
    S->pool.reset(mem_budget_bytes, 256);
    auto dev = [&](void** p, size_t b) {
        if (e == cudaSuccess) e = hh::dev_alloc(p, b);
    };
    auto host = [&](void** p, size_t b) {
        if (e == cudaSuccess) e = hh::host_alloc(p, b);
    };
    dev(reinterpret_cast<void**>(&S->jobs_dev), kJobs * sizeof(hh::ServeJob));
    dev(reinterpret_cast<void**>(&S->views_dev), kViewRecords * rec);
    dev(reinterpret_cast<void**>(&S->claimed_dev), kJobs * sizeof(unsigned));
    dev(reinterpret_cast<void**>(&S->done_dev), kJobs * sizeof(unsigned));
    dev(reinterpret_cast<void**>(&S->ctl_dev), 6 * sizeof(int));
    host(reinterpret_cast<void**>(&S->jobs_host), kJobs * sizeof(hh::ServeJob));
    host(reinterpret_cast<void**>(&S->views_host), kViewRecords * rec);
    host(reinterpret_cast<void**>(&S->pub_host), kJobs * sizeof(int));
    host(reinterpret_cast<void**>(&S->consts_host), 2 * sizeof(int));
    host(reinterpret_cast<void**>(&S->flags_host), kJobs * sizeof(unsigned));
    host(reinterpret_cast<void**>(&S->hctl_host), 2 * sizeof(int));
    if (e == cudaSuccess)
        e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&S->flags_alias), S->flags_host, 0);
    if (e == cudaSuccess)
        e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&S->hctl_alias), S->hctl_host, 0);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->ctl_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->work_stream, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&S->published, &S->worker_done, &S->reset_done})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        std::memset(S->flags_host, 0, kJobs * sizeof(unsigned));
        std::memset(S->hctl_host, 0, 2 * sizeof(int));
        S->consts_host[0] = 0;
        S->consts_host[1] = 1;
        e = cudaMemsetAsync(S->claimed_dev, 0, kJobs * sizeof(unsigned), S->work_stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(S->done_dev, 0, kJobs * sizeof(unsigned), S->work_stream);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(S->jobs_dev, 0xff, kJobs * sizeof(hh::ServeJob), S->work_stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(S->ctl_dev, 0, 6 * sizeof(int), S->work_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(S->work_stream);
    }
    if (e != cudaSuccess) {
        hh_status st = hh::cuda_fail(e, "server queue");
        hh_serve_destroy(S);
        return st;
    }
    S->stats.pool_capacity = S->pool.capacity();
    S->host_thread = std::thread([S] { S->run(); });
    *out = S;
    return hh::ok();
}

hh_status hh_serve_set_config(hh_server S, const hh_batch_config* cfg) {
    if (!S || !cfg) return hh::fail(HH_ERR_INVALID_ARG, "server or config is NULL");
    if (cfg->block_threads < 32 || cfg->block_threads > 256 || cfg->block_threads % 32 ||
        cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 64 || cfg->refill_min < 1 ||
        cfg->refill_min > 32 || (cfg->tile_w != 4 && cfg->tile_w != 8 && cfg->tile_w != 16) ||
        (cfg->tile_order != 0 && cfg->tile_order != 1) ||
        (cfg->tile_group != 0 && cfg->tile_group != 1))
        return hh::fail(HH_ERR_INVALID_ARG, "invalid launch configuration");
    std::unique_lock<std::mutex> lock(S->mu);
    // the shape is the worker's: wait (bounded) until nothing is on the GPU
    const bool idle = S->cv.wait_for(lock, std::chrono::seconds(60), [S] {
        return S->inflight.empty() && S->pending.empty();
    });
    if (!idle) return hh::fail(HH_ERR_BUSY, "requests are still running after 60 s");
    S->cfg = *cfg;
    return hh::ok();
}

hh_status hh_serve_put_volume(hh_server S, int64_t frame_id, hh_volume vol) {
    if (!S || !vol) return hh::fail(HH_ERR_INVALID_ARG, "server or volume is NULL");
    if (vol->layout != HH_LAYOUT_BRICK2)
        return hh::fail(HH_ERR_INVALID_ARG, "the volume is not a marchable (BRICK2) volume");
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
    auto fit = S->frames.find(frame_id);
    if (fit == S->frames.end())
        return hh::fail(HH_ERR_NOT_FOUND, "no frame %lld", static_cast<long long>(frame_id));
    if (S->frame_users.count(frame_id))
        return hh::fail(HH_ERR_BUSY, "frame %lld is being rendered", static_cast<long long>(frame_id));
    if (S->cls_vol == fit->second && !S->inflight.empty()) {
        // the running worker's grid was read from this volume; any volume of
        // the same grid and storage serves for a later launch
        hh_volume other = nullptr;
        for (auto& kv : S->frames)
            if (kv.first != frame_id && kv.second->nx == S->cls_vol->nx &&
                kv.second->ny == S->cls_vol->ny && kv.second->nz == S->cls_vol->nz &&
                kv.second->storage == S->cls_vol->storage)
                other = kv.second;
        if (!other)
            return hh::fail(HH_ERR_BUSY, "frame %lld gives the running requests their grid",
                            static_cast<long long>(frame_id));
        S->cls_vol = other;
    } else if (S->cls_vol == fit->second) {
        S->have_class = false;
        S->cls_vol = nullptr;
    }
    S->frames.erase(fit);
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
        r.rays += static_cast<uint64_t>(cams[i].width) * cams[i].height;
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
    if (r.state == RUNNING || r.state == PENDING)
        return hh::fail(HH_ERR_BUSY, "request %llu is not finished (cancel it first)",
                        static_cast<unsigned long long>(ticket));
    // a done request still holds its outputs (a cancelled one gave them back
    // when its tiles ended; a failed one's go back once no worker runs)
    if (r.has_memory) S->pool.release(r.offset);
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
        r.cancel_requested = true;  // its tiles finish; the result is discarded
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
    if (S->host_thread.joinable()) S->host_thread.join();
    if (S->ctl_dev && S->consts_host && S->ctl_stream) {
        S->stop_requested = false;
        S->request_stop();  // an idle worker leaves at its next poll
    }
    // the worker finishes the tiles it was given, then sees the stop request
    if (S->work_stream) cudaStreamSynchronize(S->work_stream);
    if (S->ctl_stream) cudaStreamSynchronize(S->ctl_stream);
    if (S->work_stream) cudaStreamDestroy(S->work_stream);
    if (S->ctl_stream) cudaStreamDestroy(S->ctl_stream);
    for (cudaEvent_t ev : {S->published, S->worker_done, S->reset_done})
        if (ev) cudaEventDestroy(ev);
    hh::dev_free(S->jobs_dev);
    hh::dev_free(S->views_dev);
    hh::dev_free(S->claimed_dev);
    hh::dev_free(S->done_dev);
    hh::dev_free(S->ctl_dev);
    hh::host_free(S->jobs_host);
    hh::host_free(S->views_host);
    hh::host_free(S->pub_host);
    hh::host_free(S->consts_host);
    hh::host_free(S->flags_host);
    hh::host_free(S->hctl_host);
    hh::dev_free(S->pool_base);
    delete S;
    return hh::ok();
}

}  // extern "C"
