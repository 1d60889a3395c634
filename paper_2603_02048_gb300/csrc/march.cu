// Curved-ray march (Sec. 3.3.2-3.3.3 of arXiv 2603.02048), one thread per
// pixel ray: pinhole ray generation, slab entry into the volume box, the
// march of Eq. 15 with the Eq. 16 update (or RK4) and the Eq. 18 adaptive
// step, the exit clip at the box face, and the bilinear equirect background
// at the exit direction.
//
// Precision (everything FP32, no FP64 on the device):
//  - The direction is carried as w = w_ref + d, with w_ref the primary ray
//    direction (fixed per ray) and d the small accumulated deflection. The
//    Eq. 16 normalisation is done in that form, d' = d1 + (r - 1)(w_ref + d1)
//    with r - 1 = -e / (s (1 + s)), e = 2 w_ref.d1 + |d1|^2, s = sqrt(1 + e),
//    so rounding never touches the O(1) part of w and the deflection keeps
//    full relative precision over thousands of steps.
//  - The position is a compensated pair (hi + lo): hi carries a power-of-two
//    bias B (hi = position + B, B above every coordinate and step), so every
//    increment is smaller than hi and Fast2Sum is error-free; its rounding
//    error goes to lo. The position proper is (hi - B) + lo, where hi - B is
//    exact (Sterbenz).
//  - Divisions and square roots whose operands are far from any cancellation
//    (ds / n, n theta / (|g_perp| + eps), the renormalisation term, |g_perp|)
//    use the approximate hardware forms (relative error ~1e-7, harmless next
//    to the 1e-6 rad tolerance: they perturb steps, not the path).
//
// Layout: a block of 128 threads covers a 16x8 pixel tile; each warp an 8x4
// sub-tile, so the rays of a warp stay close in the volume and their eight
// corner fetches per step share cache lines in L1. The volume is stored in
// 2x2x2 micro-bricks (BRICK2), which spreads the distinct voxels of a warp's
// corner load over all L1 bank groups.
#include "hh_internal.h"

namespace hh {
namespace {

constexpr float kPi = 3.14159265358979323846f;

struct TraceArgs {
    const void* vol;
    const float* scales;
    int nx, ny, nz;
    unsigned bx, bxy;   // BRICK2 bricks along x and per xy plane
    unsigned by8, bz8;  // BRICK2 strides (in elements) of one brick step in y and z
    float bias;         // power of two above every coordinate and step
    float3 eye, look, up;
    float vfov_deg;
    int W, H;
    float h_fixed, h_min, h_max, theta, eps;
    int max_steps;
    const uint8_t* bg;
    int bgW, bgH;
    float* rgb;
    float* exit_pos;
    float* exit_dir;
    int32_t* steps;
    uint32_t* flags;
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
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
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

// Hardware approximate square root (PTX sqrt.approx.f32, ~1 ulp).
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Lattice cell and weight along one axis: u = p - 1/2 clamped to [0, n-1],
// i0 = min(floor(u), n-2), f = u - i0. NaN positions clamp to 0.
__device__ __forceinline__ void axis_cell(float p, int n, int& i0, float& f) {
    const float u = fminf(fmaxf(p - 0.5f, 0.0f), static_cast<float>(n - 1));
    i0 = min(static_cast<int>(floorf(u)), n - 2);
    f = u - static_cast<float>(i0);
}

__device__ __forceinline__ float4 ld_fp32(const float4* __restrict__ v, unsigned i) {
    return __ldg(v + i);
}
__device__ __forceinline__ float4 ld_fp16(const ushort4* __restrict__ v, unsigned i) {
    const uint2 raw = __ldg(reinterpret_cast<const uint2*>(v) + i);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float t) {
    return make_float4(lerpf(a.x, b.x, t), lerpf(a.y, b.y, t), lerpf(a.z, b.z, t),
                       lerpf(a.w, b.w, t));
}

// Trilinear sample of {dn, g} at p (Sec. 3.3.1: n and grad n sampled with
// trilinear interpolation); FP16 volumes are interpolated as stored and
// scaled once afterwards.
template <int STORAGE>
__device__ __forceinline__ Sample fetch(const TraceArgs& A, float3 p) {
    int ix, iy, iz;
    float fx, fy, fz;
    axis_cell(p.x, A.nx, ix, fx);
    axis_cell(p.y, A.ny, iy, fy);
    axis_cell(p.z, A.nz, iz, fz);
    // BRICK2 element of corner (ix, iy, iz), then the steps to the other
    // corners: +1 in x stays in the brick (slot +1) when ix is even, else it
    // moves to the next brick (slot -1, brick +1: +7); likewise y (+2 or
    // by8 - 2) and z (+4 or bz8 - 4).
    const unsigned b = brick2_offset(ix, iy, iz, A.bx, A.bxy);
    const unsigned dx = (ix & 1) ? 7u : 1u;
    const unsigned dy = (iy & 1) ? A.by8 - 2u : 2u;
    const unsigned dz = (iz & 1) ? A.bz8 - 4u : 4u;
    const unsigned b010 = b + dy, b001 = b + dz, b011 = b001 + dy;
    float4 v000, v100, v010, v110, v001, v101, v011, v111;
    if (STORAGE == HH_STORE_FP32) {
        const float4* V = static_cast<const float4*>(A.vol);
        v000 = ld_fp32(V, b);
        v100 = ld_fp32(V, b + dx);
        v010 = ld_fp32(V, b010);
        v110 = ld_fp32(V, b010 + dx);
        v001 = ld_fp32(V, b001);
        v101 = ld_fp32(V, b001 + dx);
        v011 = ld_fp32(V, b011);
        v111 = ld_fp32(V, b011 + dx);
    } else {
        const ushort4* V = static_cast<const ushort4*>(A.vol);
        v000 = ld_fp16(V, b);
        v100 = ld_fp16(V, b + dx);
        v010 = ld_fp16(V, b010);
        v110 = ld_fp16(V, b010 + dx);
        v001 = ld_fp16(V, b001);
        v101 = ld_fp16(V, b001 + dx);
        v011 = ld_fp16(V, b011);
        v111 = ld_fp16(V, b011 + dx);
    }
    // the standard 8-corner weights
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
    const float w00 = gy * gz, w10 = fy * gz, w01 = gy * fz, w11 = fy * fz;
    const float w000 = gx * w00, w100 = fx * w00, w010 = gx * w10, w110 = fx * w10;
    const float w001 = gx * w01, w101 = fx * w01, w011 = gx * w11, w111 = fx * w11;
    float4 c;
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
    Sample s;
    if (STORAGE == HH_STORE_FP32) {
        s.dn = c.x;
        s.gx = c.y;
        s.gy = c.z;
        s.gz = c.w;
    } else {
        const float s_n = __ldg(A.scales), s_g = __ldg(A.scales + 1);
        s.dn = c.x * s_n;
        s.gx = c.y * s_g;
        s.gy = c.z * s_g;
        s.gz = c.w * s_g;
    }
    return s;
}

// Eq. 18 (second form) or the fixed step.
template <bool ADAPTIVE>
__device__ __forceinline__ float step_length(const TraceArgs& A, float n, float gperp_norm) {
    if (!ADAPTIVE) return A.h_fixed;
    return fminf(fmaxf(__fdividef(n * A.theta, gperp_norm + A.eps), A.h_min), A.h_max);
}

// Eq. 16's normalize, in deflection form: returns d' with w_ref + d' the unit
// vector along w_ref + d1 (taking |w_ref| = 1).
__device__ __forceinline__ float3 renormalize(float3 wr, float3 d1) {
    const float e = 2.0f * dot(wr, d1) + dot(d1, d1);
    const float s = sqrt_approx(1.0f + e);
    const float rm1 = __fdividef(-e, s * (1.0f + s));
    return fma3(rm1, wr + d1, d1);
}

// Colour of direction d in the equirect background (bilinear, u wraps,
// v clamps; value / 255).
__device__ __forceinline__ float3 background(const TraceArgs& A, float3 d) {
    const float phi = atan2f(d.y, d.x);
    const float theta = atan2f(sqrtf(d.x * d.x + d.y * d.y), d.z);
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

// Ray through the centre of pixel (px, py); row 0 at the top.
__device__ __forceinline__ float3 primary_ray(const TraceArgs& A, int px, int py) {
    const float3 f = normalized(A.look - A.eye);
    const float3 r = normalized(cross(f, A.up));
    const float3 u = cross(r, f);
    const float t = tanf(0.5f * A.vfov_deg * (kPi / 180.0f));
    const float W = static_cast<float>(A.W), H = static_cast<float>(A.H);
    const float a = (2.0f * (static_cast<float>(px) + 0.5f) / W - 1.0f) * t * (W / H);
    const float b = (1.0f - 2.0f * (static_cast<float>(py) + 0.5f) / H) * t;
    return normalized(fma3(b, u, fma3(a, r, f)));
}

// Slab test of o + t d against [0,nx]x[0,ny]x[0,nz]; hit iff
// t_out >= max(t_in, 0). An axis with d = 0 misses when o is outside it.
__device__ __forceinline__ bool slab(const TraceArgs& A, float3 o, float3 d, float& t_in) {
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

__device__ __forceinline__ bool outside(const TraceArgs& A, float3 p) {
    return p.x < 0.0f || p.y < 0.0f || p.z < 0.0f || p.x > static_cast<float>(A.nx) ||
           p.y > static_cast<float>(A.ny) || p.z > static_cast<float>(A.nz);
}

// Fraction tau in [0, 1] of the increment `inc` from (hi + lo) at which the
// segment leaves the box (the slab exit along the segment).
__device__ __forceinline__ float exit_fraction(const TraceArgs& A, float3 hi, float3 lo,
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

template <int STORAGE, bool ADAPTIVE>
__device__ __forceinline__ float3 perp_rate(const TraceArgs& A, float3 p, float3 w, float& n,
                                            float& gperp_norm) {
    const Sample s = fetch<STORAGE>(A, p);
    n = 1.0f + s.dn;
    const float3 g = make_float3(s.gx, s.gy, s.gz);
    const float3 gp = fma3(-dot(w, g), w, g);
    gperp_norm = sqrt_approx(dot(gp, gp));
    return gp;
}

template <int STORAGE, int STEPPER, bool ADAPTIVE>
__global__ void __launch_bounds__(128, (STEPPER == HH_STEP_RK4) ? 6 : 8) march_kernel(const TraceArgs A) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int px = blockIdx.x * 16 + (warp & 1) * 8 + (lane & 7);
    const int py = blockIdx.y * 8 + (warp >> 1) * 4 + (lane >> 3);
    if (px >= A.W || py >= A.H) return;

    const float3 wr = primary_ray(A, px, py);
    float3 ep = A.eye, ed = wr;
    uint32_t flags = 0;
    int k = 0;
    float t_in;
    if (slab(A, A.eye, wr, t_in)) {
        flags = HH_FLAG_HIT;
        // position = (hi - B) + lo with hi = position + B (see the header)
        const float B = A.bias;
        const float3 entry = fma3(fmaxf(t_in, 0.0f), wr, A.eye);
        float3 hi, lo;
        fast_two_sum(B, entry.x, hi.x, lo.x);
        fast_two_sum(B, entry.y, hi.y, lo.y);
        fast_two_sum(B, entry.z, hi.z, lo.z);
        float3 d = make_float3(0.0f, 0.0f, 0.0f);
        for (k = 0; k < A.max_steps; ++k) {
            const float3 C = make_float3((hi.x - B) + lo.x, (hi.y - B) + lo.y, (hi.z - B) + lo.z);
            float ds;
            float3 dnew, inc;
            if (STEPPER == HH_STEP_RK4) {
                float n1, gpn, n2, n3, n4, unused;
                const float3 w1 = wr + d;
                const float3 gp1 = perp_rate<STORAGE, ADAPTIVE>(A, C, w1, n1, gpn);
                ds = step_length<ADAPTIVE>(A, n1, gpn);
                const float hds = 0.5f * ds;
                const float3 k1 = __fdividef(1.0f, n1) * gp1;
                const float3 d2 = fma3(hds, k1, d);
                const float3 w2 = wr + d2;
                const float3 gp2 = perp_rate<STORAGE, ADAPTIVE>(A, fma3(hds, w1, C), w2, n2, unused);
                const float3 k2 = __fdividef(1.0f, n2) * gp2;
                const float3 d3 = fma3(hds, k2, d);
                const float3 w3 = wr + d3;
                const float3 gp3 = perp_rate<STORAGE, ADAPTIVE>(A, fma3(hds, w2, C), w3, n3, unused);
                const float3 k3 = __fdividef(1.0f, n3) * gp3;
                const float3 d4 = fma3(ds, k3, d);
                const float3 w4 = wr + d4;
                const float3 gp4 = perp_rate<STORAGE, ADAPTIVE>(A, fma3(ds, w3, C), w4, n4, unused);
                const float3 k4 = __fdividef(1.0f, n4) * gp4;
                const float3 ksum = k1 + 2.0f * (k2 + k3) + k4;
                dnew = renormalize(wr, fma3(ds * (1.0f / 6.0f), ksum, d));
                const float3 dpos = (1.0f / 6.0f) * (d + 2.0f * (d2 + d3) + d4);
                inc = ds * (wr + dpos);
            } else {
                float n, gpn;
                const float3 w = wr + d;
                const float3 gp = perp_rate<STORAGE, ADAPTIVE>(A, C, w, n, gpn);
                ds = step_length<ADAPTIVE>(A, n, gpn);
                dnew = renormalize(wr, fma3(__fdividef(ds, n), gp, d));
                inc = ds * (wr + dnew);
            }
            float3 nhi, err;
            fast_two_sum(hi.x, inc.x, nhi.x, err.x);
            fast_two_sum(hi.y, inc.y, nhi.y, err.y);
            fast_two_sum(hi.z, inc.z, nhi.z, err.z);
            const float3 nlo = lo + err;
            const float3 P = make_float3((nhi.x - B) + nlo.x, (nhi.y - B) + nlo.y,
                                         (nhi.z - B) + nlo.z);
            if (outside(A, P)) {
                const float3 h0 = make_float3(hi.x - B, hi.y - B, hi.z - B);  // exact
                const float tau = exit_fraction(A, h0, lo, inc);
                ep = h0 + fma3(tau, inc, lo);
                ed = wr + dnew;
                flags |= HH_FLAG_EXITED;
                ++k;
                break;
            }
            hi = nhi;
            lo = nlo;
            d = dnew;
        }
        if (!(flags & HH_FLAG_EXITED)) {
            flags |= HH_FLAG_MAXSTEPS;
            ep = make_float3((hi.x - B) + lo.x, (hi.y - B) + lo.y, (hi.z - B) + lo.z);
            ed = wr + d;
        }
    }
    const float3 rgb = background(A, ed);
    const size_t pix = static_cast<size_t>(py) * A.W + px;
    A.rgb[3 * pix + 0] = rgb.x;
    A.rgb[3 * pix + 1] = rgb.y;
    A.rgb[3 * pix + 2] = rgb.z;
    if (A.exit_pos) {
        A.exit_pos[3 * pix + 0] = ep.x;
        A.exit_pos[3 * pix + 1] = ep.y;
        A.exit_pos[3 * pix + 2] = ep.z;
    }
    if (A.exit_dir) {
        A.exit_dir[3 * pix + 0] = ed.x;
        A.exit_dir[3 * pix + 1] = ed.y;
        A.exit_dir[3 * pix + 2] = ed.z;
    }
    if (A.steps) A.steps[pix] = k;
    if (A.flags) A.flags[pix] = flags;
}

template <int STORAGE, int STEPPER, bool ADAPTIVE>
void launch_one(const TraceArgs& A, cudaStream_t s) {
    const dim3 block(128);
    const dim3 grid((A.W + 15) / 16, (A.H + 7) / 8);
    march_kernel<STORAGE, STEPPER, ADAPTIVE><<<grid, block, 0, s>>>(A);
}

}  // namespace

cudaError_t launch_trace(const hh_volume_s* vol, const hh_camera& cam, const hh_step_params& P,
                         const hh_background& bg, const hh_view_out& out, cudaStream_t s) {
    if (vol->layout != HH_LAYOUT_BRICK2) return cudaErrorInvalidValue;
    TraceArgs A;
    A.vol = vol->data;
    A.scales = vol->scales_dev;
    A.nx = vol->nx;
    A.ny = vol->ny;
    A.nz = vol->nz;
    A.bx = vol->bx;
    A.bxy = vol->bxy;
    A.by8 = vol->bx * 8u;
    A.bz8 = vol->bxy * 8u;
    {
        // bias: a power of two B with B >= 2 * step and B >= extent + step, so
        // positions in [-step, extent + step] keep hi in [B/2, 2B]
        const float step = P.adaptive ? P.h_max : P.h_fixed;
        const float need = fmaxf(static_cast<float>(max(vol->nx, max(vol->ny, vol->nz))) + step,
                                 2.0f * step);
        float B = 8.0f;
        while (B < need) B *= 2.0f;
        A.bias = B;
    }
    A.eye = make_float3(cam.eye[0], cam.eye[1], cam.eye[2]);
    A.look = make_float3(cam.look_at[0], cam.look_at[1], cam.look_at[2]);
    A.up = make_float3(cam.up[0], cam.up[1], cam.up[2]);
    A.vfov_deg = cam.vfov_deg;
    A.W = cam.width;
    A.H = cam.height;
    A.h_fixed = P.h_fixed;
    A.h_min = P.h_min;
    A.h_max = P.h_max;
    A.theta = P.theta_max;
    A.eps = P.eps;
    A.max_steps = P.max_steps;
    A.bg = bg.rgb8_dev;
    A.bgW = bg.width;
    A.bgH = bg.height;
    A.rgb = out.rgb;
    A.exit_pos = out.exit_pos;
    A.exit_dir = out.exit_dir;
    A.steps = out.steps;
    A.flags = out.flags;
    const bool fp16 = vol->storage == HH_STORE_FP16_SCALED;
    const bool rk4 = P.stepper == HH_STEP_RK4;
    const bool adaptive = P.adaptive != 0;
    if (!fp16 && !rk4 && !adaptive) launch_one<HH_STORE_FP32, HH_STEP_EULER_PAPER, false>(A, s);
    if (!fp16 && !rk4 && adaptive) launch_one<HH_STORE_FP32, HH_STEP_EULER_PAPER, true>(A, s);
    if (!fp16 && rk4 && !adaptive) launch_one<HH_STORE_FP32, HH_STEP_RK4, false>(A, s);
    if (!fp16 && rk4 && adaptive) launch_one<HH_STORE_FP32, HH_STEP_RK4, true>(A, s);
    if (fp16 && !rk4 && !adaptive) launch_one<HH_STORE_FP16_SCALED, HH_STEP_EULER_PAPER, false>(A, s);
    if (fp16 && !rk4 && adaptive) launch_one<HH_STORE_FP16_SCALED, HH_STEP_EULER_PAPER, true>(A, s);
    if (fp16 && rk4 && !adaptive) launch_one<HH_STORE_FP16_SCALED, HH_STEP_RK4, false>(A, s);
    if (fp16 && rk4 && adaptive) launch_one<HH_STORE_FP16_SCALED, HH_STEP_RK4, true>(A, s);
    count_launch();
    return cudaGetLastError();
}

}  // namespace hh
