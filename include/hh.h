/*
 * hh.h -- C ABI of the GB300 curved-ray heat-haze engine.
 *
 * The engine implements the rendering hot path of "Real-Time 3D Simulation of
 * Heat-Induced Air Turbulence" (arXiv 2603.02048, Sec. 3.3): SPH particle
 * densities are splatted onto a voxel grid (Sec. 3.3.1), mapped to a
 * refractive-index volume by Gladstone-Dale with its gradient by finite
 * differences (Eqs. 12-13), and one curved ray per pixel is integrated through
 * it (Eqs. 14-16) with the curvature-adaptive step of Eqs. 17-18; the exit ray
 * then sees the scene behind the volume: analytic textured planes and an
 * environment map (the stand-in for the paper's scene intersection).
 *
 * Conventions shared by every call
 *  - Units are voxels. A grid of nx*ny*nz voxels covers the box
 *    [0,nx] x [0,ny] x [0,nz]; voxel (i,j,k) has its centre at
 *    (i+1/2, j+1/2, k+1/2). Dense arrays are x-fastest:
 *    index = (k*ny + j)*nx + i.
 *  - Pointers named *_dev are CUDA device pointers on the current device; the
 *    caller owns them and keeps them alive until the work on `stream` ends.
 *    hh_volume handles are owned by the library (free with hh_volume_free).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Every call only enqueues work on it and returns; results are
 *    ready when the stream reaches that point. Calls that allocate or read
 *    back host values say so.
 *  - No call aborts, traps or prints. Each returns an hh_status; on failure
 *    hh_last_error() holds a message for the calling thread.
 *  - All arithmetic on the device is FP32 (storage may be FP16); nothing on
 *    the device uses FP64.
 */
#ifndef HH_H_
#define HH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HH_OK = 0,
    HH_ERR_INVALID_ARG = 1, /* a pointer, size or parameter is out of range */
    HH_ERR_OOM = 2,         /* device memory (or a serving budget) is short  */
    HH_ERR_CUDA = 3,        /* a CUDA runtime call failed                    */
    HH_ERR_TIMEOUT = 4,     /* a bounded wait ran out                        */
    HH_ERR_BUSY = 5,        /* the request is still running                  */
    HH_ERR_CANCELLED = 6,   /* the request was cancelled                     */
    HH_ERR_NOT_FOUND = 7    /* unknown ticket, frame or handle               */
} hh_status;

/* Storage of the {dn, grad n} volume. */
typedef enum {
    HH_STORE_FP32 = 0,       /* 4 x float per voxel, 16 B                     */
    HH_STORE_FP16_SCALED = 1 /* 4 x half per voxel, 8 B: dn / s_n and g / s_g */
} hh_storage;

/* Integrator of the ray ODE (Eq. 15). */
typedef enum {
    HH_STEP_EULER_PAPER = 0, /* Eq. 16: w' = normalize(w + ds/n g_perp), C' = C + ds w' */
    HH_STEP_RK4 = 1          /* classical RK4 of Eq. 15 in (C, w), w normalised per step  */
} hh_stepper;

/* Ray flag bits (hh_view_out.flags). */
#define HH_FLAG_HIT 1u      /* the primary ray entered the volume box          */
#define HH_FLAG_EXITED 2u   /* it left the box through the exit clip           */
#define HH_FLAG_MAXSTEPS 4u /* it used max_steps steps without leaving the box */
#define HH_FLAG_CLAMP 8u    /* HH_DEBUG_BOUNDS builds only: a trilinear corner  */
                            /* index fell outside the padded volume (clamped)  */

/* SPH particles, Sec. 3.1 Eq. 1 reduced to what the splat reads: n records of
 * float4 {x, y, z, m} on the device, positions in voxel units. */
typedef struct {
    const float* xyzm_dev;
    int64_t n;
} hh_particles;

/* Voxel grid of the refractive-index volume (Sec. 3.3.1, resolution R). */
typedef struct {
    int nx, ny, nz;  /* voxels per axis, each >= 2                            */
    float h_kernel;  /* splat smoothing length h (voxels); support radius 2h  */
    int storage;     /* hh_storage                                            */
} hh_grid;

/* Opaque library-owned volume: dn = n - 1 and grad n on the device. */
typedef struct hh_volume_s* hh_volume;

/* Pinhole camera. Pixel (x, y) has row 0 at the top; its ray passes through
 * the pixel centre: d = normalize(f + (2(x+1/2)/W - 1) t (W/H) r
 * + (1 - 2(y+1/2)/H) t u) with f = normalize(look_at - eye),
 * r = normalize(f x up), u = r x f, t = tan(vfov/2). */
typedef struct {
    float eye[3], look_at[3], up[3];
    float vfov_deg; /* vertical field of view in degrees, (0, 180) */
    int width, height;
} hh_camera;

/* Step schedule (Sec. 3.3.3). adaptive != 0: ds = clamp(n theta_max /
 * (|(I - w w^T) g| + eps), h_min, h_max) (Eq. 18, second form); otherwise
 * ds = h_fixed (the fixed-step variant of Sec. 4.1). */
typedef struct {
    int stepper;      /* hh_stepper                                          */
    int adaptive;     /* 0 or 1                                              */
    float h_fixed;    /* > 0 when !adaptive                                  */
    float h_min;      /* > 0 when adaptive                                   */
    float h_max;      /* >= h_min when adaptive                              */
    float theta_max;  /* >= 0, radians                                       */
    float eps;        /* >= 0, per voxel                                     */
    int max_steps;    /* >= 0 steps inside the box per ray                   */
} hh_step_params;

/* A textured rectangle of the scene behind or around the volume (the
 * paper's scene geometry, Sec. 4.1, in its simplest analytic form): points
 * origin + a u + b v with a, b in [0, 1]; u and v must be perpendicular and
 * non-zero. Its RGB8 texture (device, row-major H x W x 3, row 0 at b = 0) is
 * sampled bilinearly at (a W - 1/2, b H - 1/2), clamped to the texel
 * centres. Two-sided and opaque. */
typedef struct {
    float origin[3], u[3], v[3]; /* voxel units */
    const uint8_t* rgb8_dev;
    int width, height;           /* >= 2 each */
} hh_plane;

#define HH_MAX_PLANES 4

/* What a ray sees once it is straight again (after leaving the volume, or
 * from the eye when it misses it): the nearest of n_planes planes it hits in
 * front of it (t > 0), otherwise the equirectangular RGB8 environment map
 * (device, row-major H x W x 3, row 0 at the +z pole). Map colour of
 * direction d: phi = atan2(d_y, d_x), theta = polar angle from +z,
 * u = (phi/2pi + 1/2) W - 1/2, v = theta/pi H - 1/2, bilinear over texel
 * centres, u wrapping, v clamped; value/255. Planes are seen by the exit ray
 * only: the scene lies outside the refractive volume. */
typedef struct {
    const uint8_t* rgb8_dev;
    int width, height;  /* width >= 1, height >= 2 */
    int n_planes;       /* 0 .. HH_MAX_PLANES */
    hh_plane planes[HH_MAX_PLANES];
} hh_background;

/* Per-view outputs (device, caller-owned), pixel-major in row order. At
 * least one of rgb (H*W*3 floats in [0,1]) and rgb8 (H*W*3 bytes, the
 * display image: round-to-nearest-even of 255 * rgb) is required; the
 * others may be NULL. exit_pos / exit_dir: H*W*3 floats (voxel units; a ray
 * that misses the box reports the eye and its primary direction); steps:
 * H*W int32; flags: H*W uint32 of HH_FLAG_* bits. */
typedef struct {
    float* rgb;
    float* exit_pos;
    float* exit_dir;
    int32_t* steps;
    uint32_t* flags;
    uint8_t* rgb8;
} hh_view_out;

/* ---------------------------------------------------------------------- */
/* Volume construction (Sec. 3.3.1, Eqs. 12-13)                            */
/* ---------------------------------------------------------------------- */

/* Splat alone (Sec. 3.3.1): rho_dev[v] = sum_p m_p W(|x_v - x_p|, h) at voxel
 * centres, W the M4 cubic spline (support 2h). rho_dev holds nx*ny*nz floats
 * and is overwritten; voxels outside the grid are dropped. Accumulation is
 * FP32 with atomics, so the summation order (and the last bits) vary between
 * runs. grid->storage is ignored. */
hh_status hh_splat_density(const hh_particles* particles, const hh_grid* grid, float* rho_dev,
                           void* stream);

/* Gladstone-Dale + gradient (Eqs. 12-13) of a given density: dn = K_gd rho,
 * g = grad dn by central differences inside and one-sided differences on the
 * first/last voxel of each axis, stored as grid->storage. For FP16 storage
 * each value is stored as the nearest half of value / s with per-volume
 * scales s_n (for dn) and s_g (for g): the smallest powers of two with
 * max|dn| / s_n <= 16384 and max|g| / s_g <= 16384, computed on the device.
 * Allocates the volume (cudaMalloc) and returns it in *out; the computation
 * is enqueued on `stream`. */
hh_status hh_volume_from_density(const float* rho_dev, const hh_grid* grid, float K_gd,
                                 void* stream, hh_volume* out);

/* Same with dn given directly: Eq. 12's dn supplied, Eq. 13's gradient
 * computed (equivalent to K_gd = 1 on rho = dn). */
hh_status hh_volume_from_dn(const float* dn_dev, const hh_grid* grid, void* stream,
                            hh_volume* out);

/* Splat + Gladstone-Dale + gradient in one call: the full volume build of
 * Sec. 3.3.1. Allocates the volume and its density scratch (4 B/voxel, kept
 * with the volume for hh_volume_rebuild) with cudaMalloc; the computation is
 * enqueued on `stream`. */
hh_status hh_build_index_field(const hh_particles* particles, const hh_grid* grid, float K_gd,
                               void* stream, hh_volume* out);

/* Rebuilds an existing volume in place from a new particle set (the next
 * simulation frame): splat into the volume's density scratch, then Eqs.
 * 12-13, with the volume's grid, h and storage. Allocates nothing when the
 * volume came from hh_build_index_field; otherwise its first call allocates
 * the density scratch (cudaMalloc). When the density grid is larger than the
 * device's L2 cache, the particles are first sorted by cell into a
 * volume-owned copy (allocated on first use, and again when the particle
 * count grows: 16 B per particle plus 8 B per cell) so that the splat's
 * reductions stay in L2; the environment variable HH_SPLAT_SORT=0 or 1
 * forces this off or on. The result does not depend on it beyond the order
 * of the FP32 atomic sums. Work queued earlier on other streams that still
 * reads the volume must be ordered before this call by the caller. */
hh_status hh_volume_rebuild(hh_volume vol, const hh_particles* particles, float K_gd,
                            void* stream);

/* Allocation-free volume build (no counterpart in the paper: it is a service
 * for callers that cannot allocate device memory -- a host application that
 * owns the whole device-memory budget and forbids libraries from allocating,
 * or a real-time frame loop that must not pay cudaMalloc's implicit device
 * synchronisation and unbounded latency). Same computation as
 * hh_build_index_field with FP32 storage, but the density grid lives in a
 * fixed device array compiled into the library (8 MiB, held on every device
 * that loads the library until the process exits) and the result is written
 * to the caller's vol4_dev: nx*ny*nz*4 floats {dn, gx, gy, gz} per voxel,
 * x fastest (the hh_volume_export layout), 16-byte aligned.
 * - Calls no cudaMalloc, cudaFree or other allocating routine.
 * - nx*ny*nz must be at most 2,097,152 (e.g. 128^3); larger grids and
 *   grid->storage != HH_STORE_FP32 return HH_ERR_INVALID_ARG.
 * - The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 * - Every call on a device shares the one array and clears it first: calls
 *   whose work overlaps on the GPU (other streams, other host threads) race
 *   and corrupt each other's result; order them. */
hh_status hh_build_index_field_noalloc(const hh_particles* particles, const hh_grid* grid,
                                       float K_gd, float* vol4_dev, void* stream);

/* Writes the volume as the march reads it (the {dn, grad n} field of Eqs.
 * 12-13 that Sec. 3.3.1's trilinear sampling reads), dequantised to FP32,
 * into dst_dev: nx*ny*nz*4 floats {dn, gx, gy, gz} per voxel (x fastest). */
hh_status hh_volume_export(hh_volume vol, float* dst_dev, void* stream);

/* Grid, FP16 scales (1 for FP32 storage) and device bytes of a volume's
 * packed field (bookkeeping; no paper passage; the same allocation also holds
 * a free-corner mask, one bit per voxel, and its build scratch, a word per
 * stored column and 16 slices: under 5 % more). Synchronises `stream` to read
 * the scales. Any output may be NULL. */
hh_status hh_volume_info(hh_volume vol, hh_grid* grid, float* s_n, float* s_g, size_t* bytes,
                         void* stream);

/* The FP16 scales alone (1, 1 for FP32 storage; bookkeeping, no paper
 * passage): hh_volume_info on the legacy default stream. Synchronises it;
 * either output may be NULL. */
hh_status hh_volume_scales(hh_volume vol, float* s_n, float* s_g);

/* Releases the volume (cudaFree; synchronises the device first). NULL is ok.
 * Bookkeeping; no paper passage. */
hh_status hh_volume_free(hh_volume vol);

/* ---------------------------------------------------------------------- */
/* Curved-ray tracing (Sec. 3.3.2-3.3.3, Eqs. 14-18)                       */
/* ---------------------------------------------------------------------- */

/* Renders n_cams views of one volume. For every pixel: pinhole ray, slab
 * entry into the box, straight outside it; inside, per step k the volume is
 * sampled trilinearly at C_k (lattice coordinate p - 1/2 clamped to the
 * voxel centres), g_perp = (I - w w^T) g, ds by the schedule, then Eq. 16
 * (EULER_PAPER) or RK4; when a step leaves the box the segment is clipped
 * at the face and the ray leaves with the new direction. The colour is what
 * the straight ray from the exit point along the exit direction sees in `bg`
 * (its nearest textured plane, else the environment map); a ray that misses
 * the box sees it along its primary ray. outs[i] belongs to cams[i]. */
hh_status hh_trace(hh_volume vol, const hh_camera* cams, int n_cams,
                   const hh_step_params* params, const hh_background* bg,
                   const hh_view_out* outs, void* stream);

/* ---------------------------------------------------------------------- */
/* Batched multi-view launches                                             */
/* ---------------------------------------------------------------------- */

/* Many views of one volume in one persistent launch: the per-ray work is
 * hh_trace's (results are bit-identical to it), but every warp pulls
 * 32-pixel tiles of any view from one atomic counter, so views of uneven
 * size share the GPU without per-view tails. Multi-camera rendering of one
 * shared volume is the paper's scaling axis (Sec. 4.1, Table 1) and its
 * central claim (Sec. 4.2, multi-view consistency). */
typedef struct hh_batch_s* hh_batch;

/* Launch shape of a batch (hh_batch_autotune searches it). */
typedef struct {
    int block_threads; /* threads per block, a multiple of 32 in [32, 256]      */
    int blocks_per_sm; /* resident blocks per SM; 0 = the occupancy maximum     */
    int refill_min;    /* warp-level compaction: idle lanes take new pixels once
                          at least this many lanes of the warp are idle (1..32;
                          32 = only when the whole warp is idle)              */
    int tile_w;        /* pixel tile of a warp: tile_w x (32 / tile_w), 4/8/16 */
    int tile_order;    /* order in which warps take tiles: 0 = view after view,
                          row by row; 1 = the tiles of all views interleaved
                          by their relative row, so every view sweeps the
                          volume top to bottom at once (views at similar
                          elevations then share the bricks in L2: 17 % less
                          DRAM traffic on the 512^3 32-view batch).       */
    int tile_group;    /* 0 = each warp takes its own next tile; 1 = a block
                          takes one tile per warp at once (consecutive tiles,
                          neighbours in a view) so that its warps march them
                          side by side on one SM and share its L1, with a
                          barrier between groups; needs refill_min 32       */
} hh_batch_config;

/* Creates a batch of n_cams views (1..4096) over `vol` (the multi-camera
 * rendering of Sec. 4.1); outs[i] belongs to cams[i] (same layout and rules
 * as hh_trace). The library copies the view
 * table (and, for tile_order 1, the tile order) to the device (cudaMalloc +
 * synchronous copy); the volume, the background and the output buffers stay
 * owned by the caller and must outlive the batch. Default configuration:
 * {128, 0, 32, 8, 0, 0}. */
hh_status hh_batch_create(hh_volume vol, const hh_camera* cams, int n_cams,
                          const hh_step_params* params, const hh_background* bg,
                          const hh_view_out* outs, hh_batch* out);

/* Sets / reads the launch shape (a GPU scheduling choice; no paper passage).
 * Setting a new tile_w re-uploads the view table (synchronous). Get reports
 * blocks_per_sm resolved to a number. Both return HH_ERR_INVALID_ARG for a
 * NULL batch or config, set also for a shape outside the ranges above. */
hh_status hh_batch_set_config(hh_batch b, const hh_batch_config* cfg);
/* (The read half of the pair above.) */
hh_status hh_batch_get_config(hh_batch b, hh_batch_config* cfg);

/* Autotuner (a GPU scheduling search; no paper passage). Times candidate
 * configurations (tile 8x4 / 4x8 / 16x2; 64, 128, 256 threads;
 * compaction at 32, 16, 8 idle lanes; full or half occupancy; views one
 * after the other or interleaved; without compaction, warps or blocks taking
 * tiles: 144 in all) with CUDA events
 * on `stream`, each as the median of |reps| launches, and keeps the fastest.
 * Results are cached in the process by workload (grid, storage, schedule,
 * view resolutions); reps > 0 reuses a cached result, reps < 0 re-measures.
 * Synchronous; writes the outputs like a launch. */
hh_status hh_batch_autotune(hh_batch b, int reps, void* stream, hh_batch_config* best);

/* Enqueues one persistent launch (a counter reset plus one kernel) on
 * `stream`: every view's march of Secs. 3.3.2-3.3.3, as hh_trace computes it.
 * It can be captured into a CUDA graph by the caller. */
hh_status hh_batch_launch(hh_batch b, void* stream);

/* Same launch (Secs. 3.3.2-3.3.3 for every view) through a CUDA graph the
 * batch captures on its first call (on
 * `stream`, which must be a created stream, not the legacy default) and
 * replays afterwards. A new configuration or stream re-captures. */
hh_status hh_batch_launch_graph(hh_batch b, void* stream);

/* Releases the batch (its graph, view table and counter). NULL is ok.
 * Bookkeeping; no paper passage. */
hh_status hh_batch_free(hh_batch b);

/* ---------------------------------------------------------------------- */
/* Real-time frame pipeline: host particles in, host display images out    */
/* ---------------------------------------------------------------------- */

/* The per-frame loop of the paper's renderer (Sec. 3.3: each simulation
 * frame's particles splatted into the index volume, Sec. 3.3.1, then every
 * camera's view marched through it, Secs. 3.3.2-3.3.3), with the particles
 * coming from host memory and the display images (RGB8, as in hh_view_out)
 * going back to host memory. Frames are double buffered, each of the two
 * slots with its own volume, buffers and compute stream, plus an upload and
 * a download stream of the library's own: frame t+1's build runs beside
 * frame t's march, and while frame t is built and marched, frame t+1's
 * particles are uploaded and frame t-1's images downloaded, so the copies
 * overlap the kernels. One thread drives a pipeline. */
typedef struct hh_pipeline_s* hh_pipeline;

/* Creates a pipeline (the Sec. 3.3 frame loop above) for the views
 * cams[0..n_cams) (1..4096) of a volume on
 * `grid` (h_kernel > 0) with Gladstone-Dale constant K_gd, for up to
 * max_particles particles per frame. cfg NULL: one hh_trace launch per view;
 * otherwise the views run as one batched launch (hh_batch, bit-identical to
 * hh_trace) with that configuration, replayed from a CUDA graph. Allocates
 * on the current device two volumes (one per slot, with their density
 * scratch), two particle buffers and two sets of image buffers; cams and
 * params are copied; the background's device
 * buffers stay owned by the caller and must outlive the pipeline.
 * Synchronous. */
hh_status hh_pipeline_create(const hh_grid* grid, float K_gd, int64_t max_particles,
                             const hh_camera* cams, int n_cams, const hh_step_params* params,
                             const hh_background* bg, const hh_batch_config* cfg,
                             hh_pipeline* out);

/* Enqueues frame t of the Sec. 3.3 loop (its number, counting from 0, in
 * *frame): upload of the
 * n particles (float4 {x, y, z, m} in voxel units) at xyzm_host, volume
 * rebuild (hh_volume_rebuild), the march of every view, and the download of
 * view i's H*W*3 bytes to rgb8_host[i]. Returns once the frame is enqueued;
 * it first waits for frame t-2 to finish (HH_ERR_TIMEOUT after 60 s), so at
 * most two frames are in flight. The host buffers must stay valid, and
 * xyzm_host unchanged, until hh_pipeline_wait(t) returns. Page-locked host
 * memory (cudaHostAlloc) lets the copies run asynchronously; with pageable
 * memory the copies still work but block the calling thread. */
hh_status hh_pipeline_submit(hh_pipeline p, const float* xyzm_host, int64_t n,
                             uint8_t* const* rgb8_host, uint64_t* frame);

/* Waits, at most timeout_ms (HH_ERR_TIMEOUT after), until frame's images
 * are in host memory (frame bookkeeping; no paper passage). HH_ERR_NOT_FOUND for a frame not yet submitted; a
 * frame two or more behind the last submitted one is complete. */
hh_status hh_pipeline_wait(hh_pipeline p, uint64_t frame, int timeout_ms);

/* The volume of the last submitted frame's slot (bookkeeping, no paper
 * passage; owned by the pipeline, valid until hh_pipeline_free): once that
 * frame t has been waited for, it holds frame t's volume until frame t+2 is
 * submitted. */
hh_status hh_pipeline_volume(hh_pipeline p, hh_volume* vol);

/* Waits (bounded, 60 s per frame) for the submitted frames and releases the
 * pipeline; HH_ERR_TIMEOUT leaves it allocated. NULL is ok. Bookkeeping; no
 * paper passage. */
hh_status hh_pipeline_free(hh_pipeline p);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of render requests                         */
/* ---------------------------------------------------------------------- */

/* A render server for requests of 1..256 views against device-resident
 * per-simulation-frame volumes (the paper's use: many cameras observing one
 * shared, time-varying refractive volume, Sec. 1 and Sec. 4.2), with
 * ray-level continuous batching: one persistent worker kernel takes 32-pixel
 * tiles of every admitted request from a device queue that a host thread
 * appends to while it runs, so a new request's rays start as soon as warps
 * free up, beside those of the requests already on the GPU (per-ray results
 * bit-identical to hh_trace). Waiting requests are admitted smallest first
 * (fewest rays), except that one waiting over 50 ms goes ahead of all younger
 * ones, while fewer than max_slots are on the GPU and its outputs fit in the
 * server's device-memory budget; requests that do not fit yet wait (others
 * may pass them unless they have waited over 200 ms); a request whose outputs exceed
 * the whole budget is refused (HH_ERR_OOM); requests for a frame not yet put
 * wait for it. Requests with another step schedule, background or grid than
 * the running ones wait for those to finish. Every wait is bounded: the
 * host's, and the worker's (its warps leave after about 2 ms without work, and
 * the host launches it again when work arrives; a request whose queue entry
 * does not reach the device within about 5 ms of its publication fails with
 * HH_ERR_TIMEOUT instead of being waited for). */
typedef struct hh_server_s* hh_server;

/* Outputs a request asks for (rgb is always written). */
#define HH_OUT_RGB 1   /* H*W*3 floats per view                         */
#define HH_OUT_EXIT 2  /* exit_pos and exit_dir, H*W*3 floats each      */
#define HH_OUT_STEPS 4 /* steps (int32) and flags (uint32), H*W each    */
#define HH_OUT_RGB8 8  /* H*W*3 bytes per view (the display image)       */

typedef struct {
    uint64_t submitted, admitted, completed, cancelled, failed, rejected;
    uint64_t pending, running;  /* now                                      */
    uint64_t rays_completed;    /* primary rays of completed requests       */
    size_t pool_used, pool_capacity; /* bytes of the output budget         */
    uint64_t worker_launches;   /* launches of the persistent worker        */
    uint64_t worker_idle_exits; /* launches that ended by their idle limit  */
    uint64_t entry_timeouts;    /* requests failed because the worker's
                                   bounded wait for their queue entry ran
                                   out (HH_ERR_TIMEOUT)                     */
} hh_serve_stats;

/* Creates a server (the multi-camera serving above, Secs. 1 and 4.2) on the
 * current device with `mem_budget_bytes` of output memory (one cudaMalloc;
 * HH_ERR_OOM if the device cannot provide it), up to `max_slots` requests on
 * the GPU at once (1..64), its device queue (about 9 MB) and a control and a
 * worker stream. */
hh_status hh_serve_create(size_t mem_budget_bytes, int max_slots, hh_server* out);

/* Launch shape of the worker (block_threads, blocks_per_sm, tile_w of
 * hh_batch_config; refill_min, tile_order and tile_group do not apply (they
 * are checked for range only); a GPU scheduling
 * choice, no paper passage). Waits (up to 60 s, else HH_ERR_BUSY) until no
 * request is waiting or running. HH_ERR_INVALID_ARG for a shape out of
 * range. */
hh_status hh_serve_set_config(hh_server s, const hh_batch_config* cfg);

/* Registers the volume of simulation frame `frame_id` (the time-varying
 * volume of Sec. 4.2; the server borrows
 * it: its build must have finished, and it must stay alive and unchanged
 * while requests on it run; the server's streams do not wait for others). Replacing
 * or removing a frame that is being rendered returns HH_ERR_BUSY. */
hh_status hh_serve_put_volume(hh_server s, int64_t frame_id, hh_volume vol);
/* Unregisters frame `frame_id` (bookkeeping, no paper passage; the caller
 * keeps the volume):
 * HH_ERR_NOT_FOUND for an unknown frame, HH_ERR_BUSY while requests on it run. */
hh_status hh_serve_remove_volume(hh_server s, int64_t frame_id);

/* Queues a request of n_views cameras on frame `frame_id` (each view is
 * hh_trace's march of Secs. 3.3.2-3.3.3); returns its
 * ticket at once. `outputs` is a mask of HH_OUT_* bits; without HH_OUT_RGB
 * and HH_OUT_RGB8 the float image (HH_OUT_RGB) is made. */
hh_status hh_serve_submit(hh_server s, int64_t frame_id, const hh_camera* cams, int n_views,
                          const hh_step_params* params, const hh_background* bg, int outputs,
                          uint64_t* ticket);

/* Request status (bookkeeping; no paper passage): HH_OK (with the
 * submit-to-completion latency in ms) when the request is
 * done, HH_ERR_BUSY while it waits or runs, HH_ERR_CANCELLED,
 * HH_ERR_NOT_FOUND for unknown or released tickets, HH_ERR_CUDA on failure. */
hh_status hh_serve_poll(hh_server s, uint64_t ticket, double* latency_ms);

/* As poll, but waits up to timeout_ms (HH_ERR_TIMEOUT when it runs out;
 * bookkeeping, no paper passage). */
hh_status hh_serve_wait(hh_server s, uint64_t ticket, int timeout_ms, double* latency_ms);

/* Device pointers of a done request's view outputs, the march results of
 * Secs. 3.3.2-3.3.3 (inside the server's
 * budget; valid until hh_serve_release). Pixel layout as hh_view_out. */
hh_status hh_serve_view(hh_server s, uint64_t ticket, int view, hh_view_out* out);

/* Frees a finished request's outputs and forgets its ticket (bookkeeping, no
 * paper passage); a waiting or
 * running request returns HH_ERR_BUSY (cancel it first). */
hh_status hh_serve_release(hh_server s, uint64_t ticket);

/* Cancels a request (bookkeeping, no paper passage): a waiting one at once, a
 * running one when its last tile ends (its result is discarded). Cancelled
 * requests still need releasing. */
hh_status hh_serve_cancel(hh_server s, uint64_t ticket);

/* Counters of the server's life so far (hh_serve_stats; bookkeeping, no
 * paper passage). HH_ERR_INVALID_ARG for a NULL server or output. */
hh_status hh_serve_get_stats(hh_server s, hh_serve_stats* out);

/* Stops the worker, waits for running launches and frees the server
 * (bookkeeping, no paper passage). */
hh_status hh_serve_destroy(hh_server s);

/* ---------------------------------------------------------------------- */
/* Diagnostics                                                             */
/* ---------------------------------------------------------------------- */

/* Message of the last failed call on this thread ("" if none; diagnostics,
 * no paper passage). The pointer stays valid until the thread's next call. */
const char* hh_last_error(void);

/* Number of kernels this library has launched in this process (diagnostics,
 * no paper passage; graph replays count one each). */
uint64_t hh_kernel_launch_count(void);

/* Number of device (cudaMalloc) and pinned host (cudaMallocHost) buffers the
 * library holds right now, across all its objects (diagnostics, no paper
 * passage): a call that fails returns it to its value before the call. For
 * tests of the out-of-memory paths, the environment variable
 * HH_FAIL_ALLOC_AT=k makes the library's k-th allocation, counted from the
 * last change of the variable's value, fail as cudaErrorMemoryAllocation
 * (the calling entry point then returns HH_ERR_OOM); unset, nothing fails. */
int64_t hh_live_allocations(void);

/* Bounds checking of the march's volume reads (diagnostics, no paper
 * passage). A library compiled with -DHH_DEBUG_BOUNDS (the build script's
 * "debug_bounds" variant, libhh_debug_bounds.so) checks every trilinear
 * corner index of every march against the padded volume, counts those
 * outside it on the device, clamps them and sets HH_FLAG_CLAMP on the ray.
 * This call synchronises the device and returns the count in *count
 * (resetting it when `reset` is non-zero). In the normal build, which has no
 * check, it sets *count = 0 and returns HH_ERR_NOT_FOUND. */
hh_status hh_debug_bounds_violations(uint64_t* count, int reset);

#ifdef __cplusplus
}
#endif

#endif /* HH_H_ */
