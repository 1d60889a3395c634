// Curved-ray march (Sec. 3.3.2-3.3.3 of arXiv 2603.02048), one thread per
// pixel ray: pinhole ray generation, slab entry into the volume box, the
// march of Eq. 15 with the Eq. 16 update (or RK4) and the Eq. 18 adaptive
// step, the exit clip at the box face, and what the straight exit ray sees
// (textured scene planes, else the bilinear equirect environment map).
//
// Precision (everything FP32, no FP64 on the device):
//  - The direction is carried as w = w_ref + d, with w_ref the primary ray
//    direction (fixed per ray) and d the small accumulated deflection. The
//    Eq. 16 normalisation is done in that form, d' = d1 + r (w_ref + d1) with
//    1 + r = |w_ref + d1|^-1 (a Taylor polynomial in e = |w_ref + d1|^2 - 1,
//    see renormalize), so rounding never touches the O(1) part of w and the
//    deflection keeps full relative precision over thousands of steps.
//  - The position is a compensated pair (hi + lo): hi carries a power-of-two
//    bias B (hi = position + B, B above every coordinate and step), so every
//    increment is smaller than hi and Fast2Sum is error-free; its rounding
//    error goes to lo. The position proper is (hi - B) + lo, where hi - B is
//    exact (Sterbenz); the volume is sampled, and the exit tested, at the
//    lattice coordinate (hi - (B - 1/2)) + lo = position + 1/2, rounded once.
//  - Divisions and square roots whose operands are far from any cancellation
//    (ds / n, n theta / (|g_perp| + eps), the renormalisation term, |g_perp|)
//    use the approximate hardware forms (relative error ~1e-7, harmless next
//    to the 1e-6 rad tolerance: they perturb steps, not the path).
//
// Layout: a block of 128 threads covers a 16x8 pixel tile; each warp an 8x4
// sub-tile, so the rays of a warp stay close in the volume and their eight
// corner fetches per step share cache lines in L1. The volume is stored in
// 2x2x2 micro-bricks (BRICK2) with a one-voxel halo of edge copies: the
// bricks spread the distinct voxels of a warp's corner load over all L1 bank
// groups, and the halo lets a sample in the box skip every index clamp.
// A sample whose eight corners are all zero (its first corner marked in the
// volume's free-corner mask, built with the volume) is read as zero from one
// bit of that mask instead of eight brick loads, and the Eq. 16 step then
// takes n = 1, g_perp = 0 and their step length without the arithmetic (a
// warp whose lanes all sample zero skips it); every step is still taken with
// the values the general branch would compute, so the results do not depend
// on the skip.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "hh_internal.h"

namespace hh {
namespace {

constexpr float kPi = 3.14159265358979323846f;

// Resident 128-thread blocks per SM the Eq. 16 march kernels are compiled
// for: 8 leaves 64 registers per thread (measured fastest; 10 or 12 spill).
#define HH_MARCH_MIN_BLOCKS 8
// Resident 256-thread blocks per SM of the persistent batched kernel (its
// refill state needs registers beyond the single-view kernel's).
#ifndef HH_BATCH_MIN_BLOCKS
#define HH_BATCH_MIN_BLOCKS 3
#endif

// Volume-side arguments of a launch (shared by every view).
struct VolArgs {
    const void* vol;
    const float* scales;
    int nx, ny, nz;
    unsigned bx, bxy;   // BRICK2 bricks along x and per xy plane
    unsigned by8, bz8;  // BRICK2 strides (in elements) of one brick step in y and z
    unsigned long long mask_off;  // bytes from a volume's data to its free-corner mask
    float bias;         // power of two above every coordinate and step
    float bias_u;       // bias - 1/2: (hi - bias_u) + lo is the lattice coordinate
    float ux, uy, uz;   // n + 1/2: the far faces in lattice coordinates
    float h_fixed, h_min, h_max, theta, eps;
    int max_steps;
    const uint8_t* bg;
    int bgW, bgH;
    int n_planes;
    hh_plane planes[HH_MAX_PLANES];
};

// View-side arguments: the camera, the caller's output buffers and the
// view's place in a batch's tile list.
struct ViewArgs {
    float3 eye;
    float3 f, r, u;    // camera basis: forward, right, up (computed on the host in FP64)
    float a0, b0, s;   // pixel (x, y) -> a = a0 + (x + 1/2) s, b = b0 - (y + 1/2) s
    int W, H;
    float* rgb;
    uint8_t* rgb8;
    float* exit_pos;
    float* exit_dir;
    int32_t* steps;
    uint32_t* flags;
    int tiles_x;     // 8x4-pixel tiles per row
    int tile_begin;  // index of the view's first tile in the batch
};

struct Sample {
    float dn, gx, gy, gz;
};

__device__ __forceinline__ float3 operator+(float3 a, float3 b) {
    return make_float3(a.x + b.x, a.y + b.y, a.z + b.z);
}
__device__ __forceinline__ float3 operator-(float3 a, float3 b) {
    return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float3 operator*(float s, float3 a) {
    return make_float3(s * a.x, s * a.y, s * a.z);
}
// Sums of products are written with explicit FMAs: a plain a * b + c * d lets
// the compiler fuse either product, and which one it fuses follows the
// surrounding code, so results would change with unrelated edits.
__device__ __forceinline__ float dot(float3 a, float3 b) {
    return fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x));
}
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(fmaf(a.y, b.z, -(a.z * b.y)), fmaf(a.z, b.x, -(a.x * b.z)),
                       fmaf(a.x, b.y, -(a.y * b.x)));
}
__device__ __forceinline__ float3 normalized(float3 v) {
    const float len = sqrtf(dot(v, v));
    return make_float3(v.x / len, v.y / len, v.z / len);
}
// a + s * b, component-wise with FMA
__device__ __forceinline__ float3 fma3(float s, float3 b, float3 a) {
    return make_float3(fmaf(s, b.x, a.x), fmaf(s, b.y, a.y), fmaf(s, b.z, a.z));
}
__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

// Error-free sum for |a| >= |b| (Dekker's Fast2Sum): s + e == a + b exactly.
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// Packed FP32x2 (PTX fma.rn.f32x2 / sub.rn.f32x2): two FP32 lanes per
// instruction, each rounded like its scalar counterpart.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pc, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\tmov.b64 pc, {%6, %7};\n\t"
        "fma.rn.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
// a + t (b - a) on both halves of a float4 (t duplicated in tt).
__device__ __forceinline__ float4 lerp4x2(float4 a, float4 b, float2 tt) {
    const float2 lo = fma2(tt, sub2(make_float2(b.x, b.y), make_float2(a.x, a.y)),
                           make_float2(a.x, a.y));
    const float2 hi = fma2(tt, sub2(make_float2(b.z, b.w), make_float2(a.z, a.w)),
                           make_float2(a.z, a.w));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// Hardware approximate square root (PTX sqrt.approx.f32, ~1 ulp).
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Lattice cell and weight along one axis from the lattice coordinate u =
// position + 1/2, the halo coordinate of the BRICK2 layout (the centre of
// grid voxel i at u = i + 1; the march carries u, not the position):
// i0 = floor(u), f = u - i0. A position in [0, n] has u in [0.5, n + 0.5], so
// both corners i0, i0 + 1 lie in the padded axis [0, n + 1], and the halo
// copies make this the sample with the lattice coordinate clamped to the
// voxel centres. The Euler march samples only accepted points, which lie in
// the box (a NaN gives i0 = 0); CLAMP first clamps u to [0.5, n + 0.5] (NaN
// to 0.5) for RK4 stage points, which may lie outside.
template <bool CLAMP>
__device__ __forceinline__ void axis_cell(float u, int n, int& i0, float& f) {
    if (CLAMP) u = fminf(fmaxf(u, 0.5f), static_cast<float>(n) + 0.5f);
    const float fl = floorf(u);
    i0 = static_cast<int>(fl);
    f = u - fl;
}

__device__ __forceinline__ float4 ld_fp32(const float4* __restrict__ v, unsigned i) {
    return __ldg(v + i);
}
// x-lerp of two FP16 corners read raw (four halves each), in FP32: the first
// corner converted, the second converted inside the subtraction
// (sub.rn.f32.f16: one rounding, as converting first and subtracting in FP32),
// then a + t (b - a) on both channel pairs.
__device__ __forceinline__ float4 xlerp_fp16(uint2 a, uint2 b, float2 tt) {
    const float2 a0 = __half22float2(*reinterpret_cast<const __half2*>(&a.x));
    const float2 a1 = __half22float2(*reinterpret_cast<const __half2*>(&a.y));
    float2 d0, d1;
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
        "sub.rn.f32.f16 %0, l, %3;\n\tsub.rn.f32.f16 %1, h, %4;\n\t}"
        : "=f"(d0.x), "=f"(d0.y)
        : "r"(b.x), "f"(a0.x), "f"(a0.y));
    asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %2;\n\t"
        "sub.rn.f32.f16 %0, l, %3;\n\tsub.rn.f32.f16 %1, h, %4;\n\t}"
        : "=f"(d1.x), "=f"(d1.y)
        : "r"(b.y), "f"(a1.x), "f"(a1.y));
    const float2 lo = fma2(tt, d0, a0), hi = fma2(tt, d1, a1);
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// Trilinear sample of {dn, g} at lattice coordinate u = position + 1/2
// (Sec. 3.3.1: n and grad n sampled with trilinear interpolation); FP16
// volumes are interpolated as stored (code units, value / scale).
// With HH_DEBUG_BOUNDS the corner indices are checked against the padded
// axes (ix in [0, nx], so that ix + 1 <= nx + 1): a corner outside is counted
// in g_bounds_violations, flagged on the ray (HH_FLAG_CLAMP in `flags`) and
// clamped before the load. The release build has no check and no clamp.
#ifdef HH_DEBUG_BOUNDS
__device__ unsigned long long g_bounds_violations;
#endif

// Returns false, leaving s unset, for a sample whose eight corners are all
// zero (the zero sample).
template <int STORAGE, bool CLAMP>
__device__ __forceinline__ bool fetch_nonzero(const VolArgs& A, const void* __restrict__ vol,
                                              float3 u, uint32_t& flags, Sample& s) {
    int ix, iy, iz;
    float fx, fy, fz;
    axis_cell<CLAMP>(u.x, A.nx, ix, fx);
    axis_cell<CLAMP>(u.y, A.ny, iy, fy);
    axis_cell<CLAMP>(u.z, A.nz, iz, fz);
#ifdef HH_DEBUG_BOUNDS
    if (ix < 0 || ix > A.nx || iy < 0 || iy > A.ny || iz < 0 || iz > A.nz) {
        atomicAdd(&g_bounds_violations, 1ull);
        flags |= HH_FLAG_CLAMP;
        ix = min(max(ix, 0), A.nx);
        iy = min(max(iy, 0), A.ny);
        iz = min(max(iz, 0), A.nz);
        fx = fminf(fmaxf(fx, 0.0f), 1.0f);
        fy = fminf(fmaxf(fy, 0.0f), 1.0f);
        fz = fminf(fmaxf(fz, 0.0f), 1.0f);
    }
#else
    (void)flags;
#endif
    // BRICK2 element of corner (ix, iy, iz): brick b >> 3, slot b & 7.
    const unsigned b = brick2_offset(ix, iy, iz, A.bx, A.bxy);
    // A sample whose eight corners are all zero is the zero sample: read from
    // the volume's free-corner mask (bit b & 31 of word b >> 5; the funnel
    // shift takes the shift count mod 32) instead of the bricks.
    {
        const unsigned* fm =
            reinterpret_cast<const unsigned*>(static_cast<const char*>(vol) + A.mask_off);
        const unsigned w = __ldg(fm + (b >> 5));
        if (__funnelshift_r(w, w, b) & 1u) return false;
    }
    // The steps to the other corners: +1 in x stays in the brick (slot +1)
    // when ix is even, else it moves to the next brick (slot -1, brick +1:
    // +7); likewise y (+2 or by8 - 2) and z (+4 or bz8 - 4).
    const unsigned dx = (ix & 1) ? 7u : 1u;
    const unsigned dy = (iy & 1) ? A.by8 - 2u : 2u;
    const unsigned dz = (iz & 1) ? A.bz8 - 4u : 4u;
    const unsigned b010 = b + dy, b001 = b + dz, b011 = b001 + dy;
    float4 v000, v100, v010, v110, v001, v101, v011, v111;
    if (STORAGE == HH_STORE_FP32) {
        const float4* V = static_cast<const float4*>(vol);
        v000 = ld_fp32(V, b);
        v100 = ld_fp32(V, b + dx);
        v010 = ld_fp32(V, b010);
        v110 = ld_fp32(V, b010 + dx);
        v001 = ld_fp32(V, b001);
        v101 = ld_fp32(V, b001 + dx);
        v011 = ld_fp32(V, b011);
        v111 = ld_fp32(V, b011 + dx);
    }
    float4 c;
    if (STORAGE == HH_STORE_FP16_SCALED) {
    // FP16 storage: lerps along x (the second corner converted inside the
    // subtraction), then y, then z with packed FP32x2 arithmetic, two channels
    // per instruction (measured 8 % faster there; on FP32 storage the 8-weight
    // form below is faster)
    const uint2* V = static_cast<const uint2*>(vol);
    const uint2 r000 = __ldg(V + b), r100 = __ldg(V + b + dx);
    const uint2 r010 = __ldg(V + b010), r110 = __ldg(V + b010 + dx);
    const uint2 r001 = __ldg(V + b001), r101 = __ldg(V + b001 + dx);
    const uint2 r011 = __ldg(V + b011), r111 = __ldg(V + b011 + dx);
    const float2 tx = make_float2(fx, fx), ty = make_float2(fy, fy), tz = make_float2(fz, fz);
    c = lerp4x2(lerp4x2(xlerp_fp16(r000, r100, tx), xlerp_fp16(r010, r110, tx), ty),
                lerp4x2(xlerp_fp16(r001, r101, tx), xlerp_fp16(r011, r111, tx), ty), tz);
    } else {
    // the standard 8-corner weights
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
    const float w00 = gy * gz, w10 = fy * gz, w01 = gy * fz, w11 = fy * fz;
    const float w000 = gx * w00, w100 = fx * w00, w010 = gx * w10, w110 = fx * w10;
    const float w001 = gx * w01, w101 = fx * w01, w011 = gx * w11, w111 = fx * w11;
    c.x = w000 * v000.x;
    c.y = w000 * v000.y;
    c.z = w000 * v000.z;
    c.w = w000 * v000.w;
#define HH_ACC(W, V)              \
    c.x = fmaf(W, V.x, c.x);      \
    c.y = fmaf(W, V.y, c.y);      \
    c.z = fmaf(W, V.z, c.z);      \
    c.w = fmaf(W, V.w, c.w);
    HH_ACC(w100, v100)
    HH_ACC(w010, v010)
    HH_ACC(w110, v110)
    HH_ACC(w001, v001)
    HH_ACC(w101, v101)
    HH_ACC(w011, v011)
    HH_ACC(w111, v111)
#undef HH_ACC
    }
    // FP16 storage: the sample stays in code units (value / scale); the
    // power-of-two scales are applied downstream, where a product by them is
    // exact, so the result equals scaling here (see perp_of)
    s.dn = c.x;
    s.gx = c.y;
    s.gy = c.z;
    s.gz = c.w;
    return true;
}

template <int STORAGE, bool CLAMP>
__device__ __forceinline__ Sample fetch(const VolArgs& A, const void* __restrict__ vol, float3 u,
                                        uint32_t& flags) {
    Sample s;
    if (!fetch_nonzero<STORAGE, CLAMP>(A, vol, u, flags, s)) s.dn = s.gx = s.gy = s.gz = 0.0f;
    return s;
}

// Eq. 18 (second form) or the fixed step.
template <bool ADAPTIVE>
__device__ __forceinline__ float step_length(const VolArgs& A, float n, float gperp_norm) {
    if (!ADAPTIVE) return A.h_fixed;
    return fminf(fmaxf(__fdividef(n * A.theta, gperp_norm + A.eps), A.h_min), A.h_max);
}

// Eq. 16's normalize, in deflection form: returns d' with w_ref + d' the unit
// vector along w1 = w_ref + d1: w_ref + d' = (1 + r) w1 with
// 1 + r = (1 + e)^(-1/2), e = |w1|^2 - 1, r by its Taylor polynomial
// -e/2 + 3e^2/8 - 5e^3/16 (error 35 e^4 / 128). e is the squared turn of one
// step plus the previous rounding (below 1e-5 when Eq. 18 bounds the turn by
// theta_max <= 3e-3; an e below FP32 resolution rounds to 0 and leaves w1 as
// it is, as FP32 normalisation would); r only scales w1, never turns it, and
// its error is undone at the next step. Only d is carried, so the rounding of
// the update never touches the O(1) part w_ref.
__device__ __forceinline__ float renorm_term(float3 w1) {
    const float e = fmaf(w1.x, w1.x, fmaf(w1.y, w1.y, fmaf(w1.z, w1.z, -1.0f)));
    return e * fmaf(e, fmaf(-0.3125f, e, 0.375f), -0.5f);
}
__device__ __forceinline__ float3 renormalize(float3 w1, float3 d1) {
    return fma3(renorm_term(w1), w1, d1);
}

// Colour of direction d in the equirect environment map (bilinear, u wraps,
// v clamps; value / 255).
__device__ __forceinline__ float3 environment(const VolArgs& A, float3 d) {
    const float phi = atan2f(d.y, d.x);
    const float theta = atan2f(sqrtf(fmaf(d.y, d.y, d.x * d.x)), d.z);
    const float W = static_cast<float>(A.bgW), H = static_cast<float>(A.bgH);
    const float u = fmaf(phi, W / (2.0f * kPi), 0.5f * W - 0.5f);
    float v = fmaf(theta, H / kPi, -0.5f);
    const float ufl = floorf(u);
    const float fu = u - ufl;
    int i0 = static_cast<int>(ufl) % A.bgW;
    if (i0 < 0) i0 += A.bgW;
    const int i1 = (i0 + 1 == A.bgW) ? 0 : i0 + 1;
    v = fminf(fmaxf(v, 0.0f), H - 1.0f);
    const int j0 = min(static_cast<int>(floorf(v)), A.bgH - 2);
    const float fv = v - static_cast<float>(j0);
    const uint8_t* r0 = A.bg + static_cast<size_t>(j0) * A.bgW * 3;
    const uint8_t* r1 = r0 + static_cast<size_t>(A.bgW) * 3;
    float out[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float t00 = __ldg(r0 + i0 * 3 + c), t01 = __ldg(r0 + i1 * 3 + c);
        const float t10 = __ldg(r1 + i0 * 3 + c), t11 = __ldg(r1 + i1 * 3 + c);
        out[c] = lerpf(lerpf(t00, t01, fu), lerpf(t10, t11, fu), fv) * (1.0f / 255.0f);
    }
    return make_float3(out[0], out[1], out[2]);
}

__device__ __forceinline__ float3 f3(const float v[3]) { return make_float3(v[0], v[1], v[2]); }

// Bilinear RGB8 texture lookup at texel coordinates (s, t), clamped to the
// texel centres; value / 255.
__device__ __forceinline__ float3 texel_bilinear(const uint8_t* tex, int W, int H, float s,
                                                 float t) {
    s = fminf(fmaxf(s, 0.0f), static_cast<float>(W - 1));
    t = fminf(fmaxf(t, 0.0f), static_cast<float>(H - 1));
    const int i0 = min(static_cast<int>(floorf(s)), W - 2);
    const int j0 = min(static_cast<int>(floorf(t)), H - 2);
    const float fs = s - static_cast<float>(i0), ft = t - static_cast<float>(j0);
    const uint8_t* r0 = tex + (static_cast<size_t>(j0) * W + i0) * 3;
    const uint8_t* r1 = r0 + static_cast<size_t>(W) * 3;
    float out[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float t00 = __ldg(r0 + c), t01 = __ldg(r0 + 3 + c);
        const float t10 = __ldg(r1 + c), t11 = __ldg(r1 + 3 + c);
        out[c] = lerpf(lerpf(t00, t01, fs), lerpf(t10, t11, fs), ft) * (1.0f / 255.0f);
    }
    return make_float3(out[0], out[1], out[2]);
}

// What the straight ray P + t d (t > 0) sees: the nearest textured plane it
// hits, else the environment map.
// A call, not inlined: it runs once per ray, and keeping its registers out of
// the step loop's allocation is as fast as inlining it (measured).
__device__ __noinline__ float3 scene_color(const VolArgs& A, float3 P, float3 d) {
    float best_t = INFINITY, best_a = 0.0f, best_b = 0.0f;
    int best = -1;
#pragma unroll
    for (int k = 0; k < HH_MAX_PLANES; ++k) {
        if (k >= A.n_planes) break;
        const hh_plane& pl = A.planes[k];
        const float3 o = f3(pl.origin), u = f3(pl.u), v = f3(pl.v);
        const float3 nrm = cross(u, v);
        const float den = dot(d, nrm);
        if (den == 0.0f) continue;
        const float t = dot(o - P, nrm) / den;
        if (!(t > 0.0f) || !(t < best_t)) continue;
        const float3 r = fma3(t, d, P) - o;
        const float a = dot(r, u) / dot(u, u), b = dot(r, v) / dot(v, v);
        if (a >= 0.0f && a <= 1.0f && b >= 0.0f && b <= 1.0f) {
            best = k;
            best_t = t;
            best_a = a;
            best_b = b;
        }
    }
    if (best < 0) return environment(A, d);
    const uint8_t* tex = A.planes[0].rgb8_dev;
    int W = A.planes[0].width, H = A.planes[0].height;
#pragma unroll
    for (int k = 1; k < HH_MAX_PLANES; ++k)
        if (best == k) {
            tex = A.planes[k].rgb8_dev;
            W = A.planes[k].width;
            H = A.planes[k].height;
        }
    return texel_bilinear(tex, W, H, best_a * static_cast<float>(W) - 0.5f,
                          best_b * static_cast<float>(H) - 0.5f);
}

// Ray through the centre of pixel (px, py); row 0 at the top:
// normalize(f + a r + b u) with a = (2 (x + 1/2) / W - 1) t W / H and
// b = (1 - 2 (y + 1/2) / H) t, t = tan(vfov / 2), i.e. a = a0 + (x + 1/2) s,
// b = b0 - (y + 1/2) s with s = 2 t / H, a0 = -t W / H, b0 = t.
__device__ __forceinline__ float3 primary_ray(const ViewArgs& A, int px, int py) {
    const float a = fmaf(static_cast<float>(px) + 0.5f, A.s, A.a0);
    const float b = fmaf(static_cast<float>(py) + 0.5f, -A.s, A.b0);
    return normalized(fma3(b, A.u, fma3(a, A.r, A.f)));
}

// Slab test of o + t d against [0,nx]x[0,ny]x[0,nz]; hit iff
// t_out >= max(t_in, 0). An axis with d = 0 misses when o is outside it.
__device__ __forceinline__ bool slab(const VolArgs& A, float3 o, float3 d, float& t_in) {
    float tin = -INFINITY, tout = INFINITY;
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
    const float bx[3] = {static_cast<float>(A.nx), static_cast<float>(A.ny),
                         static_cast<float>(A.nz)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dd[a] == 0.0f) {
            if (oo[a] < 0.0f || oo[a] > bx[a]) return false;
            continue;
        }
        const float t1 = (0.0f - oo[a]) / dd[a];
        const float t2 = (bx[a] - oo[a]) / dd[a];
        tin = fmaxf(tin, fminf(t1, t2));
        tout = fminf(tout, fmaxf(t1, t2));
    }
    t_in = tin;
    return tout >= fmaxf(tin, 0.0f);
}

// Whether lattice coordinate u = position + 1/2 lies outside the box
// (position outside [0, n] on some axis).
__device__ __forceinline__ bool outside(const VolArgs& A, float3 u) {
    return u.x < 0.5f || u.y < 0.5f || u.z < 0.5f || u.x > A.ux || u.y > A.uy || u.z > A.uz;
}

// Fraction tau in [0, 1] of the increment `inc` from (hi + lo) at which the
// segment leaves the box (the slab exit along the segment).
__device__ __forceinline__ float exit_fraction(const VolArgs& A, float3 hi, float3 lo,
                                               float3 inc) {
    const float h3[3] = {hi.x, hi.y, hi.z}, l3[3] = {lo.x, lo.y, lo.z};
    const float i3[3] = {inc.x, inc.y, inc.z};
    const float bx[3] = {static_cast<float>(A.nx), static_cast<float>(A.ny),
                         static_cast<float>(A.nz)};
    float tau = 1.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (i3[a] > 0.0f) tau = fminf(tau, ((bx[a] - h3[a]) - l3[a]) / i3[a]);
        else if (i3[a] < 0.0f) tau = fminf(tau, ((0.0f - h3[a]) - l3[a]) / i3[a]);
    }
    return fmaxf(tau, 0.0f);
}

// n and the transverse gradient g_perp = (I - w w^T) g at u (Eq. 15), with
// |g_perp|. With FP16 storage g_perp is returned in code units, g_perp / s_g:
// the caller multiplies the scalar that scales it by s_g (gsc in ray_step). s_n
// and s_g are powers of two, so every such product is exact and the results
// equal those of scaling the sample first: n = 1 + dn s_n is one rounding
// either way, and |g_perp| = s_g |g_perp / s_g| exactly.
template <int STORAGE>
__device__ __forceinline__ float3 perp_of(const Sample& s, float3 w, float s_n, float s_g,
                                          float& n, float& gperp_norm) {
    n = STORAGE == HH_STORE_FP32 ? 1.0f + s.dn : fmaf(s.dn, s_n, 1.0f);
    const float3 g = make_float3(s.gx, s.gy, s.gz);
    const float3 gp = fma3(-dot(w, g), w, g);
    gperp_norm = sqrt_approx(dot(gp, gp));
    if (STORAGE != HH_STORE_FP32) gperp_norm *= s_g;
    return gp;
}
template <int STORAGE, bool CLAMP>
__device__ __forceinline__ float3 perp_rate(const VolArgs& A, const void* __restrict__ vol,
                                            float3 u, float3 w, float s_n, float s_g, float& n,
                                            float& gperp_norm, uint32_t& flags) {
    return perp_of<STORAGE>(fetch<STORAGE, CLAMP>(A, vol, u, flags), w, s_n, s_g, n, gperp_norm);
}

// Per-ray state of the march: primary direction w_ref, deflection d, biased
// compensated position (hi, lo) (position = (hi - B) + lo), its lattice
// coordinate rounded once, c = (hi - (B - 1/2)) + lo = position + 1/2 (where
// the volume is sampled and the exit is tested), steps taken and flags.
struct RayState {
    float3 wr, hi, lo, d, c;
    int k;
    uint32_t flags;
    float sn, sg;  // the volume's FP16 scales, read once per ray
    float ds0;     // the step length at a zero sample (n = 1, |g_perp| = 0)
};

// Pixel (x, y) of slot p (0..31) of a tile_w x (32 / tile_w) warp tile. Each
// 8-lane quarter of the warp covers a 4x2 pixel block, not a row of 8: a
// 128-bit load is served a quarter-warp at a time, and the voxels of a 4x2
// block of neighbouring rays form a 2x2 patch across the view, which falls on
// four different micro-brick slots (L1 bank groups), where a row of 8 rays
// would walk a line of voxels that alternates between two.
__device__ __forceinline__ void tile_pixel(int p, int tile_w_log2, int& x, int& y) {
    const int q = p >> 3;
    const int qx_log2 = tile_w_log2 - 2;  // quarters per tile row: 1, 2 or 4
    x = ((q & ((1 << qx_log2) - 1)) << 2) | (p & 3);
    y = ((q >> qx_log2) << 1) | ((p >> 2) & 1);
}

// Ray generation and slab entry (flags = HIT when the ray enters the box).
template <bool ADAPTIVE>
__device__ __forceinline__ void ray_begin(const VolArgs& V, const float* __restrict__ scales,
                                          const ViewArgs& C, int px, int py, RayState& R) {
    R.wr = primary_ray(C, px, py);
    R.sn = __ldg(scales);
    R.sg = __ldg(scales + 1);
    R.ds0 = step_length<ADAPTIVE>(V, 1.0f, 0.0f);
    R.k = 0;
    R.flags = 0;
    R.d = make_float3(0.0f, 0.0f, 0.0f);
    R.hi = R.lo = R.d;
    float t_in;
    if (slab(V, C.eye, R.wr, t_in)) {
        R.flags = HH_FLAG_HIT;
        // position = (hi - B) + lo with hi = position + B (see the header)
        // entry point, clamped into the box (rounding may put it just outside; the
        // march samples only positions in the box)
        float3 entry = fma3(fmaxf(t_in, 0.0f), R.wr, C.eye);
        entry.x = fminf(fmaxf(entry.x, 0.0f), static_cast<float>(V.nx));
        entry.y = fminf(fmaxf(entry.y, 0.0f), static_cast<float>(V.ny));
        entry.z = fminf(fmaxf(entry.z, 0.0f), static_cast<float>(V.nz));
        fast_two_sum(V.bias, entry.x, R.hi.x, R.lo.x);
        fast_two_sum(V.bias, entry.y, R.hi.y, R.lo.y);
        fast_two_sum(V.bias, entry.z, R.hi.z, R.lo.z);
    }
    R.c = make_float3((R.hi.x - V.bias_u) + R.lo.x, (R.hi.y - V.bias_u) + R.lo.y,
                      (R.hi.z - V.bias_u) + R.lo.z);
}

// One step of Eq. 16 (or RK4) with the Eq. 18 (or fixed) step length.
// Returns true when the step leaves the box: then ep / ed hold the exit
// point on the face and the new direction.
template <int STORAGE, int STEPPER, bool ADAPTIVE>
__device__ __forceinline__ bool ray_step(const VolArgs& V, const void* __restrict__ vol, RayState& R,
                                         float3& ep, float3& ed) {
    const float B = V.bias;
    const float3 wr = R.wr, d = R.d;
    const float3 C = R.c;
    float ds;
    float3 dnew, inc;
    const float gsc = STORAGE == HH_STORE_FP32 ? 1.0f : R.sg;  // see perp_rate
    if (STEPPER == HH_STEP_RK4) {
        float n1, gpn, n2, n3, n4, unused;
        const float3 w1 = wr + d;
        const float3 gp1 = perp_rate<STORAGE, true>(V, vol, C, w1, R.sn, R.sg, n1, gpn, R.flags);
        ds = step_length<ADAPTIVE>(V, n1, gpn);
        const float hds = 0.5f * ds;
        const float3 k1 = (__fdividef(1.0f, n1) * gsc) * gp1;
        const float3 d2 = fma3(hds, k1, d);
        const float3 w2 = wr + d2;
        const float3 gp2 = perp_rate<STORAGE, true>(V, vol, fma3(hds, w1, C), w2, R.sn, R.sg, n2,
                                                    unused, R.flags);
        const float3 k2 = (__fdividef(1.0f, n2) * gsc) * gp2;
        const float3 d3 = fma3(hds, k2, d);
        const float3 w3 = wr + d3;
        const float3 gp3 = perp_rate<STORAGE, true>(V, vol, fma3(hds, w2, C), w3, R.sn, R.sg, n3,
                                                    unused, R.flags);
        const float3 k3 = (__fdividef(1.0f, n3) * gsc) * gp3;
        const float3 d4 = fma3(ds, k3, d);
        const float3 w4 = wr + d4;
        const float3 gp4 = perp_rate<STORAGE, true>(V, vol, fma3(ds, w3, C), w4, R.sn, R.sg, n4,
                                                    unused, R.flags);
        const float3 k4 = (__fdividef(1.0f, n4) * gsc) * gp4;
        // k1 + 2 (k2 + k3) + k4 (every k is a product: the adds are kept
        // unfused, __fadd_rn, so no product is folded into them)
        const float3 ksum =
            make_float3(__fadd_rn(fmaf(2.0f, __fadd_rn(k2.x, k3.x), k1.x), k4.x),
                        __fadd_rn(fmaf(2.0f, __fadd_rn(k2.y, k3.y), k1.y), k4.y),
                        __fadd_rn(fmaf(2.0f, __fadd_rn(k2.z, k3.z), k1.z), k4.z));
        const float3 dsum = fma3(ds * (1.0f / 6.0f), ksum, d);
        dnew = renormalize(wr + dsum, dsum);
        const float3 dpos = (1.0f / 6.0f) * (d + 2.0f * (d2 + d3) + d4);
        inc = ds * (wr + dpos);
    } else {
        Sample smp;
        float3 d1;
        if (fetch_nonzero<STORAGE, false>(V, vol, C, R.flags, smp)) {
            float n, gpn;
            const float3 gp = perp_of<STORAGE>(smp, wr + d, R.sn, R.sg, n, gpn);
            ds = step_length<ADAPTIVE>(V, n, gpn);
            d1 = fma3(__fdividef(ds, n) * gsc, gp, d);
        } else {
            // the zero sample: n = 1 and g_perp = 0 exactly, so the branch
            // above would give the step length ds0 (the same operations on
            // the same operands) and d1 = d + 0 = d (d is never -0: it starts
            // at +0 and a sum that rounds to zero is +0); a warp whose lanes
            // all sample zero skips the g_perp and Eq. 18 arithmetic
            ds = R.ds0;
            d1 = d;
        }
        // Eq. 16: w' = normalize(w1), C' = C + ds w'; with w' = (1 + r) w1
        // the increment is ds (1 + r) w1 (w' itself is formed only at the exit)
        const float3 w1 = wr + d1;
        const float rm1 = renorm_term(w1);
        dnew = fma3(rm1, w1, d1);
        inc = fmaf(ds, rm1, ds) * w1;
    }
    float3 nhi, err;
    fast_two_sum(R.hi.x, inc.x, nhi.x, err.x);
    fast_two_sum(R.hi.y, inc.y, nhi.y, err.y);
    fast_two_sum(R.hi.z, inc.z, nhi.z, err.z);
    const float3 nlo = R.lo + err;
    const float Bu = V.bias_u;
    const float3 P = make_float3((nhi.x - Bu) + nlo.x, (nhi.y - Bu) + nlo.y, (nhi.z - Bu) + nlo.z);
    ++R.k;
    const float3 ohi = R.hi, olo = R.lo;
    R.hi = nhi;
    R.lo = nlo;
    R.c = P;
    R.d = dnew;
    if (outside(V, P)) {
        const float3 h0 = make_float3(ohi.x - B, ohi.y - B, ohi.z - B);  // exact
        const float tau = exit_fraction(V, h0, olo, inc);
        ep = h0 + fma3(tau, inc, olo);
        ed = wr + dnew;
        R.flags |= HH_FLAG_EXITED;
        return true;
    }
    return false;
}

// Display byte of a colour in [0, 1]: round-to-nearest-even of 255 v.
__device__ __forceinline__ uint8_t to_u8(float v) {
    return static_cast<uint8_t>(__float2uint_rn(__fmul_rn(fminf(fmaxf(v, 0.0f), 1.0f), 255.0f)));
}

// Final state, background lookup and the writes of one pixel. A ray that
// missed reports the eye and its primary direction; one that ran out of
// steps reports its current state (MAXSTEPS).
__device__ __forceinline__ void ray_end(const VolArgs& V, const ViewArgs& C, int px, int py,
                                        const RayState& R, float3 ep, float3 ed) {
    uint32_t flags = R.flags;
    if (!(flags & HH_FLAG_HIT)) {
        ep = C.eye;
        ed = R.wr;
    } else if (!(flags & HH_FLAG_EXITED)) {
        flags |= HH_FLAG_MAXSTEPS;
        ep = make_float3((R.hi.x - V.bias) + R.lo.x, (R.hi.y - V.bias) + R.lo.y,
                         (R.hi.z - V.bias) + R.lo.z);
        ed = R.wr + R.d;
    }
    const float3 rgb = scene_color(V, ep, ed);
    const size_t pix = static_cast<size_t>(py) * C.W + px;
    if (C.rgb) {
        C.rgb[3 * pix + 0] = rgb.x;
        C.rgb[3 * pix + 1] = rgb.y;
        C.rgb[3 * pix + 2] = rgb.z;
    }
    if (C.rgb8) {
        C.rgb8[3 * pix + 0] = to_u8(rgb.x);
        C.rgb8[3 * pix + 1] = to_u8(rgb.y);
        C.rgb8[3 * pix + 2] = to_u8(rgb.z);
    }
    if (C.exit_pos) {
        C.exit_pos[3 * pix + 0] = ep.x;
        C.exit_pos[3 * pix + 1] = ep.y;
        C.exit_pos[3 * pix + 2] = ep.z;
    }
    if (C.exit_dir) {
        C.exit_dir[3 * pix + 0] = ed.x;
        C.exit_dir[3 * pix + 1] = ed.y;
        C.exit_dir[3 * pix + 2] = ed.z;
    }
    if (C.steps) C.steps[pix] = R.k;
    if (C.flags) C.flags[pix] = flags;
}

// One view, one thread per pixel: a block of 128 threads covers 16x8 pixels,
// each warp an 8x4 tile.
template <int STORAGE, int STEPPER, bool ADAPTIVE>
__global__ void __launch_bounds__(128, (STEPPER == HH_STEP_RK4) ? 6 : HH_MARCH_MIN_BLOCKS)
    march_kernel(const VolArgs V, const ViewArgs C) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int tx, ty;
    tile_pixel(lane, 3, tx, ty);
    const int px = blockIdx.x * 16 + (warp & 1) * 8 + tx;
    const int py = blockIdx.y * 8 + (warp >> 1) * 4 + ty;
    if (px >= C.W || py >= C.H) return;
    RayState R;
    float3 ep = C.eye, ed = C.eye;
    ray_begin<ADAPTIVE>(V, V.scales, C, px, py, R);
    if (R.flags & HH_FLAG_HIT)
        while (R.k < V.max_steps && !ray_step<STORAGE, STEPPER, ADAPTIVE>(V, V.vol, R, ep, ed)) {
        }
    ray_end(V, C, px, py, R, ep, ed);
}

// View and view-local index of batch tile t: from the order table when
// there is one (tiles of all views in the order the table gives), else the
// last view whose first tile is <= t (views one after the other).
__device__ __forceinline__ void tile_of(int t, int n_views, const int* s_begin,
                                        const uint2* __restrict__ order, int& view,
                                        int& local) {
    if (order) {
        const uint2 o = __ldg(order + t);
        view = static_cast<int>(o.x);
        local = static_cast<int>(o.y);
        return;
    }
    int lo = 0, hi = n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_begin[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    view = lo;
    local = t - s_begin[lo];
}

// Persistent batched march over many views of uneven size. Each warp pulls
// 32-pixel tiles (tile_w x 32/tile_w pixels) of any view from one atomic
// counter and marches them lane by lane. Warp-level compaction: when at
// least refill_min lanes are idle (their rays left the volume, missed it or
// ran out of steps), the idle lanes take the next pixels of the warp's
// current tile (and of the next tile when it runs out) while the other lanes
// keep marching; refill_min = 32 refills only when every lane is idle, i.e.
// plain tile-at-a-time scheduling, compiled separately (REFILL = false) as
// march_kernel's loop around a tile counter. In that mode `group` = 1 makes
// the block, not the warp, the unit of scheduling: one atomic fetches one
// tile per warp (consecutive tiles: neighbours in a view), the block's warps
// march them side by side on one SM, sharing its L1, and meet at a barrier
// before the next group, as march_kernel's blocks do when they retire. The
// per-ray arithmetic is march_kernel's.
template <int STORAGE, int STEPPER, bool ADAPTIVE, bool REFILL>
__global__ void __launch_bounds__(256, (STEPPER == HH_STEP_RK4) ? 3 : HH_BATCH_MIN_BLOCKS)
    march_batch_kernel(const VolArgs V, const ViewArgs* __restrict__ views, int n_views,
                       int total_tiles, int tile_w, unsigned* __restrict__ counter,
                       int refill_min, const uint2* __restrict__ order, int group) {
    extern __shared__ int s_begin[];  // first tile of each view, then total_tiles
    for (int i = threadIdx.x; i <= n_views; i += blockDim.x)
        s_begin[i] = i < n_views ? views[i].tile_begin : total_tiles;
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int tile_w_log2 = tile_w == 16 ? 4 : (tile_w == 8 ? 3 : 2);
    if (!REFILL) {
        __shared__ int s_group;  // first tile of the block's current group
        const int warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
        int lx, ly;
        tile_pixel(lane, tile_w_log2, lx, ly);
        for (;;) {
            int t = 0;
            if (group) {  // block-uniform branch
                if (threadIdx.x == 0) s_group = static_cast<int>(atomicAdd(counter, 1u)) * warps;
                __syncthreads();
                const int g0 = s_group;
                __syncthreads();  // read by every warp before thread 0 writes it again
                if (g0 >= total_tiles) return;
                t = g0 + warp;
                if (t >= total_tiles) continue;
            } else {
                if (lane == 0) t = static_cast<int>(atomicAdd(counter, 1u));
                t = __shfl_sync(FULL, t, 0);
                if (t >= total_tiles) return;
            }
            int lo, local;
            tile_of(t, n_views, s_begin, order, lo, local);
            const ViewArgs& C = views[lo];
            const int ty = local / C.tiles_x, tx = local - ty * C.tiles_x;
            const int px = (tx << tile_w_log2) + lx, py = ty * (32 >> tile_w_log2) + ly;
            if (px < C.W && py < C.H) {
                RayState R;
                float3 ep = make_float3(0.0f, 0.0f, 0.0f), ed = ep;
                ray_begin<ADAPTIVE>(V, V.scales, C, px, py, R);
                if (R.flags & HH_FLAG_HIT)
                    while (R.k < V.max_steps && !ray_step<STORAGE, STEPPER, ADAPTIVE>(V, V.vol, R, ep, ed)) {
                    }
                ray_end(V, C, px, py, R, ep, ed);
            }
        }
    }
    int tile_local = 0, tile_view = 0, pos = 32;  // the warp's pixel stream (warp-uniform)
    bool done = false, have = false;
    int vi = 0, px = 0, py = 0;
    RayState R;
    float3 ep = make_float3(0.0f, 0.0f, 0.0f), ed = ep;
    for (;;) {
        const unsigned free_mask = __ballot_sync(FULL, !have);
        if (!done && __popc(free_mask) >= refill_min) {
            unsigned todo = free_mask;
            while (todo && !done) {
                if (pos >= 32) {
                    int t = 0;
                    if (lane == 0) t = static_cast<int>(atomicAdd(counter, 1u));
                    t = __shfl_sync(FULL, t, 0);
                    if (t >= total_tiles) {
                        done = true;
                        break;
                    }
                    tile_of(t, n_views, s_begin, order, tile_view, tile_local);
                    pos = 0;
                }
                const int avail = 32 - pos;
                const int rank = __popc(todo & lt_mask);
                const bool mine = ((todo >> lane) & 1u) && rank < avail;
                if (mine) {
                    const ViewArgs& C = views[tile_view];
                    const int local = tile_local;
                    const int p = pos + rank;
                    const int ty = local / C.tiles_x, tx = local - ty * C.tiles_x;
                    int lx, ly;
                    tile_pixel(p, tile_w_log2, lx, ly);
                    px = (tx << tile_w_log2) + lx;
                    py = ty * (32 >> tile_w_log2) + ly;
                    vi = tile_view;
                    if (px < C.W && py < C.H) {
                        ray_begin<ADAPTIVE>(V, V.scales, C, px, py, R);
                        if ((R.flags & HH_FLAG_HIT) && V.max_steps > 0) have = true;
                        else ray_end(V, C, px, py, R, ep, ed);
                    }
                }
                pos += min(avail, __popc(todo));
                todo &= ~__ballot_sync(FULL, mine);
            }
        }
        if (__ballot_sync(FULL, have) == 0u) {
            if (done) break;
            continue;
        }
        if (have) {
            if (ray_step<STORAGE, STEPPER, ADAPTIVE>(V, V.vol, R, ep, ed) || R.k >= V.max_steps) {
                ray_end(V, views[vi], px, py, R, ep, ed);
                have = false;
            }
        }
    }
}

// The render server's persistent worker (ray-level continuous batching):
// jobs (requests) are published by the host into a device queue while the
// kernel runs. A warp keeps a cursor j on the job table: it waits for job j
// to be published (n_jobs > j) and written (its entry's seq == j), takes
// tiles of it from the job's counter until they run out, then moves on. The
// warp that finishes a job's last tile raises the job's flag in host-mapped
// memory. Every wait is bounded in time (the global nanosecond timer): a warp
// whose queue has stayed empty for idle_ns counts itself idle, and once every
// warp of the launch is idle they all leave together (a warp that finds work
// again uncounts itself; the host launches the worker again when new work
// arrives, so the whole grid, not a remnant of it, serves the next burst); a
// warp told to stop leaves when idle; and a job whose entry does not appear
// within entry_ns of its publication being seen is failed (flag
// HH_JOB_FAILED) instead of waited for. Idle polls back off
// from 1 to 32 us, so thousands of idle warps do not crowd the queue's cache
// line. The per-ray arithmetic is march_kernel's (ray_begin / ray_step /
// ray_end) on the volume of the tile's job.
__device__ __forceinline__ int ld_acquire_int(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                 : "=r"(old)
                 : "l"(p), "r"(v)
                 : "memory");
    return old;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Resident 256-thread blocks per SM of the serving worker: 4 (64 registers)
// for the Eq. 16 march, whose per-tile and per-job state lives outside the
// step loop.
#ifndef HH_WORKER_MIN_BLOCKS
#define HH_WORKER_MIN_BLOCKS 4
#endif

template <int STORAGE, int STEPPER, bool ADAPTIVE>
__global__ void __launch_bounds__(256, (STEPPER == HH_STEP_RK4) ? 3 : HH_WORKER_MIN_BLOCKS)
    serve_worker_kernel(const VolArgs V, const ServeWorkerArgs W) {
    extern __shared__ __align__(16) unsigned char s_raw[];  // one view record per warp
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ViewArgs& C = reinterpret_cast<ViewArgs*>(s_raw)[warp];
    const int tile_w_log2 = W.tile_w == 16 ? 4 : (W.tile_w == 8 ? 3 : 2);
    const int tile_h = 32 >> tile_w_log2;
    int lx, ly;
    tile_pixel(lane, tile_w_log2, lx, ly);
    const char* views = static_cast<const char*>(W.views);
    constexpr int kWords = sizeof(ViewArgs) / sizeof(unsigned);
    int j = ld_acquire_int(W.first_open);
    int have_job = -1;
    int view_first = 0, view_end = 0;  // job-relative tiles of the view in C
    const void* jvol = nullptr;
    const float* jscales = nullptr;
    int jview_begin = 0, jn_views = 0, jn_tiles = 0;
    unsigned t = 0;  // this warp's claimed tile of job j (valid while have_job == j)
    bool claimed_next = false;
    unsigned long long idle_since = 0;
    unsigned backoff = 1000;
    bool counted_idle = false;
    if (lane == 0) atomicAdd(W.started_warps, 1);
    for (;;) {
        if (j != have_job) {
            // wait for job j: published, then written (both bounded in time)
            int ok = 0;
            if (lane == 0) {
                if (j < ld_acquire_int(W.n_jobs)) {
                    ok = 1;
                    if (*reinterpret_cast<const volatile unsigned*>(W.claimed + j) >=
                        HH_JOB_CLAIM_FAILED) {
                        ok = 2;  // failed by another warp: skip it
                    } else if (ld_acquire_int(&W.jobs[j].seq) != j) {
                        const unsigned long long t0 = global_ns();
                        while (ld_acquire_int(&W.jobs[j].seq) != j) {
                            if (global_ns() - t0 > W.entry_ns) {
                                ok = 2;
                                if (atomicOr(W.claimed + j, HH_JOB_CLAIM_FAILED) <
                                    HH_JOB_CLAIM_FAILED) {
                                    __threadfence_system();
                                    W.host_done[j] = HH_JOB_FAILED;
                                }
                                break;
                            }
                            __nanosleep(1000);
                        }
                    }
                } else if (ld_acquire_int(W.stop) != 0) {
                    ok = -1;  // stop requested
                }
            }
            ok = __shfl_sync(FULL, ok, 0);
            if (ok == -1) {
                if (lane == 0) W.host_ctl[1] = HH_WORKER_STOPPED;
                break;
            }
            if (ok == 0) {  // nothing published beyond j: idle (bounded)
                int leave = 0;
                if (lane == 0) {
                    const unsigned long long now = global_ns();
                    if (idle_since == 0) idle_since = now;
                    if (!counted_idle && now - idle_since > W.idle_ns) {
                        counted_idle = true;
                        // all warps that have started are idle: the launch leaves
                        // (a block that starts later sees the flag and leaves too)
                        if (atomicAdd(W.idle_warps, 1) + 1 == ld_acquire_int(W.started_warps))
                            atomicExch(W.leave, 1);
                    }
                    leave = ld_acquire_int(W.leave);
                }
                if (__shfl_sync(FULL, leave, 0)) break;
                __nanosleep(backoff);
                backoff = min(backoff * 2u, 32000u);
                j = max(j, ld_acquire_int(W.first_open));
                continue;
            }
            if (ok == 2) {
                ++j;
                continue;
            }
            idle_since = 0;
            backoff = 1000;
            if (counted_idle) {
                if (lane == 0) atomicSub(W.idle_warps, 1);
                counted_idle = false;
            }
            const ServeJob* e = W.jobs + j;
            jvol = reinterpret_cast<const void*>(
                __ldcg(reinterpret_cast<const unsigned long long*>(&e->vol)));
            jscales = reinterpret_cast<const float*>(
                __ldcg(reinterpret_cast<const unsigned long long*>(&e->scales)));
            jview_begin = __ldcg(&e->view_begin);
            jn_views = __ldcg(&e->n_views);
            jn_tiles = __ldcg(&e->n_tiles);
            have_job = j;
            view_first = view_end = 0;
            claimed_next = false;
        }
        if (!claimed_next) {
            if (lane == 0) t = atomicAdd(W.claimed + j, 1u);
            t = __shfl_sync(FULL, t, 0);
        }
        claimed_next = false;
        if (t >= static_cast<unsigned>(jn_tiles)) {  // exhausted (or failed): next job
            ++j;
            if (lane == 0) atomicMax(W.first_open, j);
            continue;
        }
        const int ti = static_cast<int>(t);
        if (ti < view_first || ti >= view_end) {
            // the tile's view: the last view of the job whose first tile is <= t
            int lo = 0, hi = jn_views - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                const ViewArgs* vm = reinterpret_cast<const ViewArgs*>(
                    views + static_cast<size_t>(jview_begin + mid) * sizeof(ViewArgs));
                if (__ldcg(&vm->tile_begin) <= ti) lo = mid;
                else hi = mid - 1;
            }
            __syncwarp();
            const unsigned* src = reinterpret_cast<const unsigned*>(
                views + static_cast<size_t>(jview_begin + lo) * sizeof(ViewArgs));
            for (int w = lane; w < kWords; w += 32) reinterpret_cast<unsigned*>(&C)[w] = __ldcg(src + w);
            __syncwarp();
            view_first = C.tile_begin;
            view_end = view_first + C.tiles_x * ((C.H + tile_h - 1) / tile_h);
        }
        const int local = ti - view_first;
        const int ty = local / C.tiles_x, tx = local - ty * C.tiles_x;
        const int px = (tx << tile_w_log2) + lx, py = ty * tile_h + ly;
        if (px < C.W && py < C.H) {
            RayState R;
            float3 ep = make_float3(0.0f, 0.0f, 0.0f), ed = ep;
            ray_begin<ADAPTIVE>(V, jscales, C, px, py, R);
            if (R.flags & HH_FLAG_HIT)
                while (R.k < V.max_steps && !ray_step<STORAGE, STEPPER, ADAPTIVE>(V, jvol, R, ep, ed)) {
                }
            ray_end(V, C, px, py, R, ep, ed);
        }
        // count the tile (release: its outputs are ordered before the count,
        // so the warp that sees the count reach n_tiles sees every tile) and
        // claim the next one in the same breath, unless the launch is leaving
        // (then the next launch takes the job's remaining tiles)
        __syncwarp();
        unsigned next = 0;
        int leave = 0;
        if (lane == 0) {
            const unsigned before = atom_add_acq_rel(W.done + j, 1u);
            leave = ld_acquire_int(W.leave);
            if (!leave) next = atomicAdd(W.claimed + j, 1u);
            if (before + 1u == static_cast<unsigned>(jn_tiles)) {
                __threadfence_system();
                W.host_done[j] = HH_JOB_DONE;
            }
        }
        if (__shfl_sync(FULL, leave, 0)) break;
        t = __shfl_sync(FULL, next, 0);
        claimed_next = true;
    }
}

template <int STORAGE, int STEPPER, bool ADAPTIVE>
void launch_one(const VolArgs& V, const ViewArgs& C, cudaStream_t s) {
    const dim3 block(128);
    const dim3 grid((C.W + 15) / 16, (C.H + 7) / 8);
    march_kernel<STORAGE, STEPPER, ADAPTIVE><<<grid, block, 0, s>>>(V, C);
}

// Calls F<STORAGE, STEPPER, ADAPTIVE>::run(args...) for the runtime choice.
template <template <int, int, bool> class F, typename... Args>
void dispatch(int storage, int stepper, int adaptive, Args&&... args) {
    const bool fp16 = storage == HH_STORE_FP16_SCALED, rk4 = stepper == HH_STEP_RK4;
    if (!fp16 && !rk4 && !adaptive) F<HH_STORE_FP32, HH_STEP_EULER_PAPER, false>::run(args...);
    if (!fp16 && !rk4 && adaptive) F<HH_STORE_FP32, HH_STEP_EULER_PAPER, true>::run(args...);
    if (!fp16 && rk4 && !adaptive) F<HH_STORE_FP32, HH_STEP_RK4, false>::run(args...);
    if (!fp16 && rk4 && adaptive) F<HH_STORE_FP32, HH_STEP_RK4, true>::run(args...);
    if (fp16 && !rk4 && !adaptive) F<HH_STORE_FP16_SCALED, HH_STEP_EULER_PAPER, false>::run(args...);
    if (fp16 && !rk4 && adaptive) F<HH_STORE_FP16_SCALED, HH_STEP_EULER_PAPER, true>::run(args...);
    if (fp16 && rk4 && !adaptive) F<HH_STORE_FP16_SCALED, HH_STEP_RK4, false>::run(args...);
    if (fp16 && rk4 && adaptive) F<HH_STORE_FP16_SCALED, HH_STEP_RK4, true>::run(args...);
}

template <int ST, int SP, bool AD>
struct SingleLaunch {
    static void run(const VolArgs& V, const ViewArgs& C, cudaStream_t s) {
        launch_one<ST, SP, AD>(V, C, s);
    }
};

// refill_min >= 32 runs the tile-at-a-time instantiation (REFILL = false).
template <int ST, int SP, bool AD>
struct BatchLaunch {
    static void run(const VolArgs& V, const ViewArgs* views, int n_views, int total_tiles,
                    int tile_w, unsigned* counter, int refill_min, const uint2* order, int group,
                    int blocks, int threads, cudaStream_t s) {
        const size_t smem = (n_views + 1) * sizeof(int);
        if (refill_min >= 32)
            march_batch_kernel<ST, SP, AD, false><<<blocks, threads, smem, s>>>(
                V, views, n_views, total_tiles, tile_w, counter, refill_min, order, group);
        else
            march_batch_kernel<ST, SP, AD, true><<<blocks, threads, smem, s>>>(
                V, views, n_views, total_tiles, tile_w, counter, refill_min, order, 0);
    }
};

template <int ST, int SP, bool AD>
struct WorkerLaunch {
    static void run(const VolArgs& V, const ServeWorkerArgs& W, int blocks, int threads,
                    cudaStream_t s) {
        const size_t smem = (threads / 32) * sizeof(ViewArgs);
        serve_worker_kernel<ST, SP, AD><<<blocks, threads, smem, s>>>(V, W);
    }
};

template <int ST, int SP, bool AD>
struct WorkerOccupancy {
    static void run(int threads, int* blocks_per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, serve_worker_kernel<ST, SP, AD>,
                                                      threads, (threads / 32) * sizeof(ViewArgs));
    }
};

template <int ST, int SP, bool AD>
struct BatchOccupancy {
    static void run(int threads, size_t smem, int refill_min, int* blocks_per_sm) {
        if (refill_min >= 32)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                blocks_per_sm, march_batch_kernel<ST, SP, AD, false>, threads, smem);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                blocks_per_sm, march_batch_kernel<ST, SP, AD, true>, threads, smem);
    }
};

VolArgs make_vol_args(const hh_volume_s* vol, const hh_step_params& P, const hh_background& bg) {
    VolArgs A;
    A.vol = vol->data;
    A.scales = vol->scales_dev;
    A.nx = vol->nx;
    A.ny = vol->ny;
    A.nz = vol->nz;
    A.bx = vol->bx;
    A.bxy = vol->bxy;
    A.by8 = vol->bx * 8u;
    A.bz8 = vol->bxy * 8u;
    A.mask_off = vol->bytes;
    // bias: a power of two B with B >= 2 * step and B >= extent + step + 1, so
    // positions in [-step, extent + step] keep hi in [B/2, 2B - 1] and both
    // hi - B and hi - (B - 1/2) are exact (Sterbenz)
    const float step = P.adaptive ? P.h_max : P.h_fixed;
    const float need =
        fmaxf(static_cast<float>(max(vol->nx, max(vol->ny, vol->nz))) + step + 1.0f, 2.0f * step);
    float B = 8.0f;
    while (B < need) B *= 2.0f;
    A.bias = B;
    A.bias_u = B - 0.5f;
    A.ux = static_cast<float>(vol->nx) + 0.5f;
    A.uy = static_cast<float>(vol->ny) + 0.5f;
    A.uz = static_cast<float>(vol->nz) + 0.5f;
    A.h_fixed = P.h_fixed;
    A.h_min = P.h_min;
    A.h_max = P.h_max;
    A.theta = P.theta_max;
    A.eps = P.eps;
    A.max_steps = P.max_steps;
    A.bg = bg.rgb8_dev;
    A.bgW = bg.width;
    A.bgH = bg.height;
    A.n_planes = bg.n_planes;
    for (int k = 0; k < HH_MAX_PLANES; ++k) A.planes[k] = bg.planes[k];
    return A;
}

ViewArgs make_view_args(const hh_camera& cam, const hh_view_out& out, int tile_w) {
    ViewArgs C;
    C.eye = make_float3(cam.eye[0], cam.eye[1], cam.eye[2]);
    // camera basis and pixel mapping, once per view in FP64 (see primary_ray)
    double f[3], r[3], u[3], fn = 0.0, rn = 0.0;
    for (int a = 0; a < 3; ++a) {
        f[a] = static_cast<double>(cam.look_at[a]) - cam.eye[a];
        fn += f[a] * f[a];
    }
    for (int a = 0; a < 3; ++a) f[a] /= std::sqrt(fn);
    const double up[3] = {cam.up[0], cam.up[1], cam.up[2]};
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    for (int a = 0; a < 3; ++a) rn += r[a] * r[a];
    for (int a = 0; a < 3; ++a) r[a] /= std::sqrt(rn);
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    C.f = make_float3(static_cast<float>(f[0]), static_cast<float>(f[1]), static_cast<float>(f[2]));
    C.r = make_float3(static_cast<float>(r[0]), static_cast<float>(r[1]), static_cast<float>(r[2]));
    C.u = make_float3(static_cast<float>(u[0]), static_cast<float>(u[1]), static_cast<float>(u[2]));
    const double t = std::tan(0.5 * static_cast<double>(cam.vfov_deg) * (M_PI / 180.0));
    C.a0 = static_cast<float>(-t * cam.width / cam.height);
    C.b0 = static_cast<float>(t);
    C.s = static_cast<float>(2.0 * t / cam.height);
    C.W = cam.width;
    C.H = cam.height;
    C.rgb = out.rgb;
    C.rgb8 = out.rgb8;
    C.exit_pos = out.exit_pos;
    C.exit_dir = out.exit_dir;
    C.steps = out.steps;
    C.flags = out.flags;
    C.tiles_x = (cam.width + tile_w - 1) / tile_w;
    C.tile_begin = 0;
    return C;
}
}  // namespace

cudaError_t launch_trace(const hh_volume_s* vol, const hh_camera& cam, const hh_step_params& P,
                         const hh_background& bg, const hh_view_out& out, cudaStream_t s) {
    if (vol->layout != HH_LAYOUT_BRICK2) return cudaErrorInvalidValue;
    const VolArgs V = make_vol_args(vol, P, bg);
    const ViewArgs C = make_view_args(cam, out, 8);
    dispatch<SingleLaunch>(vol->storage, P.stepper, P.adaptive, V, C, s);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hh

namespace hh {

size_t view_record_bytes() { return sizeof(ViewArgs); }

int build_view_table(const hh_camera* cams, const hh_view_out* outs, int n, int tile_w,
                     void* host_records) {
    ViewArgs* v = static_cast<ViewArgs*>(host_records);
    const int tile_h = 32 / tile_w;
    int64_t tiles = 0;
    for (int i = 0; i < n; ++i) {
        v[i] = make_view_args(cams[i], outs[i], tile_w);
        v[i].tile_begin = static_cast<int>(tiles);
        tiles += static_cast<int64_t>(v[i].tiles_x) * ((cams[i].height + tile_h - 1) / tile_h);
        if (tiles > (int64_t(1) << 30)) return -1;
    }
    return static_cast<int>(tiles);
}

int serve_worker_blocks_per_sm(int storage, int stepper, int adaptive, int threads) {
    int bps = 0;
    dispatch<WorkerOccupancy>(storage, stepper, adaptive, threads, &bps);
    return max(bps, 1);
}

cudaError_t launch_serve_worker(const hh_volume_s* like, const hh_step_params& P,
                                const hh_background& bg, const ServeWorkerArgs& W, int blocks,
                                int threads, cudaStream_t s) {
    if (like->layout != HH_LAYOUT_BRICK2) return cudaErrorInvalidValue;
    const VolArgs V = make_vol_args(like, P, bg);
    dispatch<WorkerLaunch>(like->storage, P.stepper, P.adaptive, V, W, blocks, threads, s);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hh

// ------------------------------------------------------------------------
// Batched multi-view launches (hh_batch_*)
// ------------------------------------------------------------------------
struct hh_batch_s {
    hh_volume vol = nullptr;
    hh_step_params params{};
    hh_background bg{};
    std::vector<hh_camera> cams;
    std::vector<hh_view_out> outs;
    hh_batch_config cfg{};
    int total_tiles = 0;
    hh::ViewArgs* views_dev = nullptr;
    unsigned* counter_dev = nullptr;
    uint2* order_dev = nullptr;  // tile order table (NULL: views one after the other)
    int sm_count = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;
};

namespace {

using hh::fail;
using hh::cuda_fail;

void drop_graph(hh_batch b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_stream = nullptr;
}

// The interleaved tile order (tile_order 1): the tiles of all views sorted by
// their relative row in their view (then by view, then by column), so that
// every view sweeps the volume top to bottom at the same time.
std::vector<uint2> interleaved_order(const std::vector<hh::ViewArgs>& v, int tile_w) {
    struct Key {
        double k;
        uint32_t view, local;
    };
    std::vector<Key> keys;
    const int tile_h = 32 / tile_w;
    for (size_t i = 0; i < v.size(); ++i) {
        const int tiles_y = (v[i].H + tile_h - 1) / tile_h;
        for (int ty = 0; ty < tiles_y; ++ty)
            for (int tx = 0; tx < v[i].tiles_x; ++tx)
                keys.push_back({(ty + 0.5) / tiles_y, static_cast<uint32_t>(i),
                                static_cast<uint32_t>(ty * v[i].tiles_x + tx)});
    }
    std::stable_sort(keys.begin(), keys.end(), [](const Key& x, const Key& y) { return x.k < y.k; });
    std::vector<uint2> ord(keys.size());
    for (size_t j = 0; j < keys.size(); ++j) ord[j] = make_uint2(keys[j].view, keys[j].local);
    return ord;
}

// Uploads the view table for the current tile width (synchronous).
hh_status upload_views(hh_batch b) {
    std::vector<hh::ViewArgs> v(b->cams.size());
    int tiles = 0;
    const int tile_w = b->cfg.tile_w, tile_h = 32 / tile_w;
    for (size_t i = 0; i < v.size(); ++i) {
        v[i] = hh::make_view_args(b->cams[i], b->outs[i], tile_w);
        v[i].tile_begin = tiles;
        const int64_t t = static_cast<int64_t>(v[i].tiles_x) * ((b->cams[i].height + tile_h - 1) / tile_h);
        if (tiles + t > (int64_t(1) << 30)) return fail(HH_ERR_INVALID_ARG, "batch has too many pixels");
        tiles += static_cast<int>(t);
    }
    b->total_tiles = tiles;
    cudaError_t e = cudaMemcpy(b->views_dev, v.data(), v.size() * sizeof(hh::ViewArgs),
                               cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "uploading the view table");
    hh::dev_free(b->order_dev);
    b->order_dev = nullptr;
    if (b->cfg.tile_order == 1) {
        std::vector<uint2> ord = interleaved_order(v, tile_w);
        e = hh::dev_alloc(reinterpret_cast<void**>(&b->order_dev), ord.size() * sizeof(uint2));
        if (e == cudaSuccess)
            e = cudaMemcpy(b->order_dev, ord.data(), ord.size() * sizeof(uint2),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "uploading the tile order");
    }
    return HH_OK;
}

hh_status check_config(const hh_batch_config* c) {
    if (!c) return fail(HH_ERR_INVALID_ARG, "config is NULL");
    if (c->block_threads < 32 || c->block_threads > 256 || c->block_threads % 32)
        return fail(HH_ERR_INVALID_ARG, "block_threads must be a multiple of 32 in [32, 256]");
    if (c->blocks_per_sm < 0 || c->blocks_per_sm > 64)
        return fail(HH_ERR_INVALID_ARG, "blocks_per_sm must be in [0, 64]");
    if (c->refill_min < 1 || c->refill_min > 32)
        return fail(HH_ERR_INVALID_ARG, "refill_min must be in [1, 32]");
    if (c->tile_w != 4 && c->tile_w != 8 && c->tile_w != 16)
        return fail(HH_ERR_INVALID_ARG, "tile_w must be 4, 8 or 16");
    if (c->tile_order != 0 && c->tile_order != 1)
        return fail(HH_ERR_INVALID_ARG, "tile_order must be 0 or 1");
    if (c->tile_group != 0 && c->tile_group != 1)
        return fail(HH_ERR_INVALID_ARG, "tile_group must be 0 or 1");
    if (c->tile_group == 1 && c->refill_min != 32)
        return fail(HH_ERR_INVALID_ARG, "tile_group 1 needs tile-at-a-time scheduling (refill_min 32)");
    return HH_OK;
}

int resident_blocks(hh_batch b, int threads, int refill_min) {
    int bps = 0;
    const size_t smem = (b->cams.size() + 1) * sizeof(int);
    hh::dispatch<hh::BatchOccupancy>(b->vol->storage, b->params.stepper, b->params.adaptive,
                                     threads, smem, refill_min, &bps);
    return std::max(bps, 1);
}

int grid_blocks(hh_batch b) {
    const int bps = b->cfg.blocks_per_sm > 0
                        ? b->cfg.blocks_per_sm
                        : resident_blocks(b, b->cfg.block_threads, b->cfg.refill_min);
    return b->sm_count * bps;
}

// Counter reset + one persistent launch of `blocks` blocks (no host queries,
// so it can run inside a stream capture).
cudaError_t enqueue(hh_batch b, int blocks, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b->counter_dev, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const int threads = b->cfg.block_threads;
    const hh::VolArgs V = hh::make_vol_args(b->vol, b->params, b->bg);
    hh::dispatch<hh::BatchLaunch>(b->vol->storage, b->params.stepper, b->params.adaptive, V,
                                  b->views_dev, static_cast<int>(b->cams.size()), b->total_tiles,
                                  b->cfg.tile_w, b->counter_dev, b->cfg.refill_min,
                                  static_cast<const uint2*>(b->order_dev), b->cfg.tile_group,
                                  blocks, threads, s);
    hh::count_launch();
    return cudaGetLastError();
}

// Autotuner results by workload signature (grid, storage, schedule, views).
std::mutex g_tune_mutex;
std::map<std::string, hh_batch_config> g_tune_cache;

std::string signature(hh_batch b) {
    std::string k = std::to_string(b->vol->nx) + "x" + std::to_string(b->vol->ny) + "x" +
                    std::to_string(b->vol->nz) + "/" + std::to_string(b->vol->storage) + "/" +
                    std::to_string(b->params.stepper) + std::to_string(b->params.adaptive);
    for (const auto& c : b->cams) k += "/" + std::to_string(c.width) + "x" + std::to_string(c.height);
    return k;
}

}  // namespace

extern "C" {

hh_status hh_batch_create(hh_volume vol, const hh_camera* cams, int n_cams,
                          const hh_step_params* params, const hh_background* bg,
                          const hh_view_out* outs, hh_batch* out) {
    if (!out) return fail(HH_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!vol) return fail(HH_ERR_INVALID_ARG, "volume is NULL");
    if (n_cams < 1 || n_cams > 4096 || !cams || !outs)
        return fail(HH_ERR_INVALID_ARG, "a batch needs 1 to 4096 cameras and outputs");
    hh_status st = hh::check_params(params);
    if (st != HH_OK) return st;
    if ((st = hh::check_background(bg)) != HH_OK) return st;
    for (int i = 0; i < n_cams; ++i) {
        if ((st = hh::check_camera(cams[i], i)) != HH_OK) return st;
        if (!outs[i].rgb && !outs[i].rgb8)
            return fail(HH_ERR_INVALID_ARG, "view %d: rgb and rgb8 outputs are both NULL", i);
    }
    hh_batch b = new (std::nothrow) hh_batch_s();
    if (!b) return fail(HH_ERR_OOM, "host allocation failed");
    b->vol = vol;
    b->params = *params;
    b->bg = *bg;
    b->cams.assign(cams, cams + n_cams);
    b->outs.assign(outs, outs + n_cams);
    b->cfg = hh_batch_config{128, 0, 32, 8, 0, 0};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = hh::dev_alloc(reinterpret_cast<void**>(&b->views_dev), n_cams * sizeof(hh::ViewArgs));
    if (e == cudaSuccess) e = hh::dev_alloc(reinterpret_cast<void**>(&b->counter_dev), sizeof(unsigned));
    if (e != cudaSuccess) {
        hh::dev_free(b->views_dev);
        delete b;
        return cuda_fail(e, "batch allocation");
    }
    if ((st = upload_views(b)) != HH_OK) {
        hh_batch_free(b);
        return st;
    }
    *out = b;
    return hh::ok();
}

hh_status hh_batch_set_config(hh_batch b, const hh_batch_config* cfg) {
    if (!b) return fail(HH_ERR_INVALID_ARG, "batch is NULL");
    hh_status st = check_config(cfg);
    if (st != HH_OK) return st;
    const bool retile = cfg->tile_w != b->cfg.tile_w || cfg->tile_order != b->cfg.tile_order;
    b->cfg = *cfg;
    drop_graph(b);
    if (retile && (st = upload_views(b)) != HH_OK) return st;
    return hh::ok();
}

hh_status hh_batch_get_config(hh_batch b, hh_batch_config* cfg) {
    if (!b || !cfg) return fail(HH_ERR_INVALID_ARG, "batch or config is NULL");
    *cfg = b->cfg;
    if (cfg->blocks_per_sm == 0)
        cfg->blocks_per_sm = resident_blocks(b, b->cfg.block_threads, b->cfg.refill_min);
    return hh::ok();
}

hh_status hh_batch_launch(hh_batch b, void* stream) {
    if (!b) return fail(HH_ERR_INVALID_ARG, "batch is NULL");
    cudaError_t e = enqueue(b, grid_blocks(b), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    return hh::ok();
}

hh_status hh_batch_launch_graph(hh_batch b, void* stream) {
    if (!b) return fail(HH_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!s) return fail(HH_ERR_INVALID_ARG, "graph launches need a created (non-default) stream");
    if (b->exec && b->graph_stream != s) drop_graph(b);
    if (!b->exec) {
        const int blocks = grid_blocks(b);
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "begin capture");
        cudaError_t le = enqueue(b, blocks, s);
        e = cudaStreamEndCapture(s, &b->graph);
        if (le != cudaSuccess) {
            drop_graph(b);
            return cuda_fail(le, "batch launch during capture");
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) {
            drop_graph(b);
            return cuda_fail(e, "graph capture");
        }
        b->graph_stream = s;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    hh::count_launch();
    return hh::ok();
}

hh_status hh_batch_autotune(hh_batch b, int reps, void* stream, hh_batch_config* best) {
    if (!b) return fail(HH_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const std::string key = signature(b);
    if (reps > 0) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            hh_status st = hh_batch_set_config(b, &it->second);
            if (st == HH_OK && best) *best = it->second;
            return st;
        }
    }
    if (reps == 0) return fail(HH_ERR_INVALID_ARG, "reps must be non-zero");
    const int n = reps < 0 ? -reps : reps;
    std::vector<hh_batch_config> cand;
    for (int to : {0, 1})
        for (int tw : {8, 4, 16})
            for (int th : {128, 256, 64})
                for (int rm : {32, 16, 8})
                    for (int bps : {0, -2})
                        for (int tg : {0, 1})
                            if (tg == 0 || rm == 32)
                                cand.push_back(hh_batch_config{th, bps, rm, tw, to, tg});
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    hh_batch_config best_cfg = b->cfg;
    hh_status st = HH_OK;
    for (auto c : cand) {
        if (c.blocks_per_sm < 0)
            c.blocks_per_sm = std::max(1, resident_blocks(b, c.block_threads, c.refill_min) / 2);
        if ((st = hh_batch_set_config(b, &c)) != HH_OK) break;
        std::vector<float> t;
        const int blocks = grid_blocks(b);
        cudaError_t e = enqueue(b, blocks, s);  // warm-up
        for (int r = 0; r < n && e == cudaSuccess; ++r) {
            cudaEventRecord(e0, s);
            e = enqueue(b, blocks, s);
            cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            t.push_back(ms);
        }
        if (e != cudaSuccess) {
            st = cuda_fail(e, "autotune trial");
            break;
        }
        std::sort(t.begin(), t.end());
        const float med = t[t.size() / 2];
        if (med < best_ms) {
            best_ms = med;
            best_cfg = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HH_OK) return st;
    if ((st = hh_batch_set_config(b, &best_cfg)) != HH_OK) return st;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = best_cfg;
    }
    if (best) *best = best_cfg;
    return hh::ok();
}

hh_status hh_debug_bounds_violations(uint64_t* count, int reset) {
    if (!count) return fail(HH_ERR_INVALID_ARG, "count is NULL");
#ifdef HH_DEBUG_BOUNDS
    unsigned long long c = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&c, hh::g_bounds_violations, sizeof c);
    if (e == cudaSuccess && reset) {
        const unsigned long long zero = 0;
        e = cudaMemcpyToSymbol(hh::g_bounds_violations, &zero, sizeof zero);
    }
    if (e != cudaSuccess) return cuda_fail(e, "reading the bounds counter");
    *count = c;
    return hh::ok();
#else
    (void)reset;
    *count = 0;
    return fail(HH_ERR_NOT_FOUND, "this library was built without HH_DEBUG_BOUNDS");
#endif
}

hh_status hh_batch_free(hh_batch b) {
    if (!b) return hh::ok();
    drop_graph(b);
    hh::dev_free(b->views_dev);
    hh::dev_free(b->counter_dev);
    hh::dev_free(b->order_dev);
    delete b;
    return hh::ok();
}

}  // extern "C"
