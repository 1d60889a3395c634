// Internal declarations shared by the C-ABI layer (api.cpp) and the kernels.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "hh.h"

// FP16 storage scales a channel group by the smallest power of two that maps
// its largest |value| to at most this code (so to more than half of it), and
// every value down to ~7e-9 of the maximum is a normal half.
#define HH_FP16_CODE_MAX 16384.0f

// Volume layouts.
//  LINEAR: x fastest, index (k*ny + j)*nx + i (the export / interchange layout).
//  BRICK2: 2x2x2 micro-bricks over the grid with a one-voxel halo: voxel
//          (i,j,k) sits at padded coordinates (I,J,K) = (i+1, j+1, k+1), and
//          the halo (I = 0 or n+1 on some axis) holds a copy of the nearest
//          grid voxel, so a trilinear sample clamped to the edge needs no
//          index clamps. Brick (I>>1, J>>1, K>>1) in x-fastest order over
//          ceil((n+2)/2) bricks per axis; inside a brick the voxel sits at
//          slot (I&1) | (J&1)<<1 | (K&1)<<2. One FP32 brick is one 128-byte
//          line, and the eight corners of any trilinear cell occupy eight
//          different slots, i.e. eight different 16-byte L1 bank groups, so a
//          warp's corner loads spread over all banks whatever the view
//          direction (the linear layout puts every y/z neighbour of a
//          power-of-two grid into the same bank group).
enum { HH_LAYOUT_LINEAR = 0, HH_LAYOUT_BRICK2 = 1 };

// Bricks along an axis of n voxels in the BRICK2 layout (halo included).
__host__ __device__ __forceinline__ unsigned brick2_count(int n) {
    return static_cast<unsigned>((n + 3) / 2);
}

// Element of padded coordinates (I, J, K) in the BRICK2 layout.
__host__ __device__ __forceinline__ unsigned brick2_offset(unsigned i, unsigned j, unsigned k,
                                                           unsigned bx, unsigned bxy) {
    return (((k >> 1) * bxy + (j >> 1) * bx + (i >> 1)) << 3) | ((k & 1u) << 2) |
           ((j & 1u) << 1) | (i & 1u);
}


struct hh_volume_s {
    int nx, ny, nz;
    int storage;        // hh_storage
    int layout;         // HH_LAYOUT_*
    unsigned bx, bxy;   // BRICK2: bricks along x, bricks per xy plane
    float h_kernel;
    void* data;         // float4 (FP32) or ushort4 of halves (FP16) per voxel
    size_t bytes;       // bytes of data (BRICK2: halo of one voxel, axes padded to even)
    // BRICK2 free-corner mask, one bit per stored element in the layout's own
    // order (bit b & 31 of word b >> 5 for element b), at data + bytes in the
    // same allocation: set when the element's voxel and its +1 neighbours on
    // each axis hold no stored nonzero value, so that a sample whose first
    // corner is that voxel reads eight zeros. Null for LINEAR volumes.
    unsigned bz;           // bricks along z
    size_t mask_words;     // 32-bit words of the mask
    unsigned* free_dev;
    uint32_t* colbits_dev; // scratch of the mask build: a word per stored column and z run
    float* scales_dev;  // [2] = {s_n, s_g} on the device (1, 1 for FP32)
    unsigned* max_dev;  // [2] = bit patterns of max|dn|, max|g| (FP16 build)
    float* rho_dev;     // density scratch for particle builds (nullable)
    float4* sorted_dev; // particles binned by cell, for grids larger than L2 (nullable)
    int64_t sorted_cap; // particles sorted_dev holds
    unsigned* bins_dev; // 2 x bin count counters of the binning (nullable)
    int n_bins;         // bins of bins_dev
    int device;
};

namespace hh {

extern std::atomic<uint64_t> g_launches;

inline void count_launch(uint64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Error reporting shared by the C-ABI entry points (defined in api.cpp): set
// the calling thread's hh_last_error() message and return the status.
hh_status fail(hh_status st, const char* fmt, ...);
hh_status cuda_fail(cudaError_t e, const char* what);
hh_status ok();

// Device (cudaMalloc) and pinned host (cudaMallocHost) allocations of the
// library, counted; HH_FAIL_ALLOC_AT=k fails the k-th one (defined in
// api.cpp). The free functions accept NULL.
cudaError_t dev_alloc(void** p, size_t bytes);
void dev_free(void* p);
cudaError_t host_alloc(void** p, size_t bytes);
void host_free(void* p);
int64_t live_allocations();

// Argument checks shared by the trace entry points (defined in api.cpp).
hh_status check_params(const hh_step_params* P);
hh_status check_camera(const hh_camera& c, int i);
hh_status check_background(const hh_background* bg);

// Kernel launchers. Each returns the launch status (cudaGetLastError()).
cudaError_t launch_splat(const float4* xyzm, int64_t n, int nx, int ny, int nz, float h,
                         float* rho, cudaStream_t s);

// Counting sort of particles by cubic cell (splat_bin_count bins, x-fastest)
// into `sorted` (n float4), using `bins` (2 x splat_bin_count unsigned) as
// counters; the splat of the sorted copy keeps its reductions within a few
// cells at a time.
int splat_bin_count(int nx, int ny, int nz);
cudaError_t launch_bin_particles(const float4* xyzm, int64_t n, int nx, int ny, int nz,
                                 unsigned* bins, float4* sorted, cudaStream_t s);

cudaError_t launch_field(const float* rho, int nx, int ny, int nz, float K, hh_volume_s* vol,
                         cudaStream_t s);

cudaError_t launch_export(const hh_volume_s* vol, float4* dst, cudaStream_t s);

// View records for a caller-managed device view table (the server's jobs):
// build_view_table fills n records of view_record_bytes() each in host memory
// for tile width tile_w and returns the total tile count (-1 if too many).
size_t view_record_bytes();
int build_view_table(const hh_camera* cams, const hh_view_out* outs, int n, int tile_w,
                     void* host_records);

// The render server's persistent worker (ray-level continuous batching).
// The host publishes requests ("jobs") into a device queue while the worker
// runs; its warps take 32-pixel tiles of the oldest job that still has some,
// and the warp that finishes a job's last tile raises the job's flag in
// host-mapped memory. Jobs are numbered from 0 since the queue's last reset;
// the host resets the queue only while no worker runs.
struct ServeJob {
    const void* vol;      // the frame's volume data (BRICK2)
    const float* scales;  // its FP16 scales on the device
    int view_begin;       // first record of the job in the view table
    int n_views;
    int n_tiles;          // tiles of all its views (view tile_begin is job-relative)
    int seq;              // the job's number; a slot holding another number is not written yet
};

// Exit reasons of a worker launch (host_ctl[1]).
enum { HH_WORKER_IDLE = 1, HH_WORKER_STOPPED = 2 };
// Values of a job's host flag.
enum { HH_JOB_DONE = 1, HH_JOB_FAILED = 2 };

struct ServeWorkerArgs {
    const ServeJob* jobs;       // job table (device)
    const void* views;          // view records (device), view_record_bytes() apart
    unsigned* claimed;          // per job: tiles handed out (from HH_JOB_CLAIM_FAILED up: failed)
    unsigned* done;             // per job: tiles finished
    const int* n_jobs;          // jobs published (device; written by host copies)
    int* first_open;            // lowest job that may still have tiles to hand out
    const int* stop;            // non-zero: leave when idle (device; written by a host copy)
    int* idle_warps;            // warps of this launch that count themselves idle
    int* leave;                 // set once every started warp is idle: the launch leaves
    int* started_warps;         // warps of this launch that have started (all three zeroed per launch)
    volatile unsigned* host_done;  // per job, host-mapped: HH_JOB_DONE / HH_JOB_FAILED
    volatile int* host_ctl;     // host-mapped: [1] exit reason
    int tile_w;
    unsigned long long idle_ns;   // a warp leaves after this long with an empty queue
    unsigned long long entry_ns;  // a published job's entry missing this long fails it
};
// A failed job's claim counter is ORed with this bit: every later claim then
// reads as beyond the job's tiles (jobs hold fewer than 2^30 tiles, and fewer
// than 2^31 claims follow).
#define HH_JOB_CLAIM_FAILED 0x80000000u

// Resident blocks per SM of the worker for a launch shape, and its launch
// (VolArgs from `like`: dims, storage, schedule, background; the volume data
// and scales come from each job).
int serve_worker_blocks_per_sm(int storage, int stepper, int adaptive, int threads);
cudaError_t launch_serve_worker(const hh_volume_s* like, const hh_step_params& P,
                                const hh_background& bg, const ServeWorkerArgs& W, int blocks,
                                int threads, cudaStream_t s);

cudaError_t launch_trace(const hh_volume_s* vol, const hh_camera& cam,
                         const hh_step_params& P, const hh_background& bg,
                         const hh_view_out& out, cudaStream_t s);

}  // namespace hh
