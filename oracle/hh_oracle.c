/*
 * hh_oracle.c -- plain FP64 CPU oracle for the curved-ray heat-haze hot path
 * of "Real-Time 3D Simulation of Heat-Induced Air Turbulence" (arXiv 2603.02048).
 *
 * TEST INFRASTRUCTURE ONLY. This file is compiled into oracle/liboracle.so and
 * is loaded by tests/, by __graft_entry__.smoke() and by the CPU-baseline leg
 * of bench.py. The CUDA library never links, includes or calls it, and it
 * includes nothing of the CUDA library: the two share no code.
 *
 * Everything is double precision and written as plain loops in the order the
 * paper states the method. There is no blocking, fusion or reordering. Each
 * function names the passage it restates; where the paper is silent, the
 * reading taken is written next to the code.
 *
 * Units: positions, step lengths and gradients are in voxel units. The grid
 * covers the box [0,nx] x [0,ny] x [0,nz]; voxel (i,j,k) has its centre at
 * (i+1/2, j+1/2, k+1/2); arrays are x-fastest: idx = (k*ny + j)*nx + i.
 *
 * Parity: every function here is pinned by tests/test_oracle_pins.py against
 * closed forms, invariants or brute force (no function is "parity unpinned").
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HHO_PI 3.14159265358979323846

/* flag bits of a traced ray */
#define HHO_FLAG_HIT 1u       /* the ray entered the volume box            */
#define HHO_FLAG_EXITED 2u    /* it left the box through the exit clip     */
#define HHO_FLAG_MAXSTEPS 4u  /* it ran out of steps inside the box        */

/* ------------------------------------------------------------------------- */
/* small vector helpers                                                       */
/* ------------------------------------------------------------------------- */
static double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double a[3], const double b[3], double out[3]) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}
static void normalize3(double v[3]) {
    double len = sqrt(dot3(v, v));
    v[0] /= len;
    v[1] /= len;
    v[2] /= len;
}

/* ------------------------------------------------------------------------- */
/* Splat (Sec. 3.3.1): rho(x_v) = sum_p m_p W(|x_v - x_p|, h) at voxel centres */
/* ------------------------------------------------------------------------- */

/*
 * M4 cubic-spline smoothing kernel in 3D, q = r/h, support 2h:
 *   W = 1/(pi h^3) * (1 - 3/2 q^2 + 3/4 q^3)   for 0 <= q < 1
 *     = 1/(pi h^3) * 1/4 (2 - q)^3             for 1 <= q < 2
 *     = 0                                      otherwise.
 * The paper names no splat kernel (Sec. 3.3.1 says "SPH kernel splatting");
 * the M4 spline is the reading taken (it is the standard SPH density kernel).
 */
double hho_kernel_m4(double r, double h) {
    double q = r / h;
    double norm = 1.0 / (HHO_PI * h * h * h);
    if (q < 1.0) return norm * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
    if (q < 2.0) {
        double t = 2.0 - q;
        return norm * 0.25 * t * t * t;
    }
    return 0.0;
}

/*
 * Density of n particles (xyzm: n x {x, y, z, m}, FP32 as the caller stores
 * them, widened exactly to FP64 here) at every voxel centre. Voxels outside
 * the grid are dropped. The sum runs particle by particle over the voxels
 * whose centres lie within 2h on every axis (W is zero beyond 2h).
 */
void hho_splat(const float* xyzm, int64_t n, int nx, int ny, int nz, double h, double* rho) {
    int dims[3] = {nx, ny, nz};
    memset(rho, 0, sizeof(double) * (size_t)nx * ny * nz);
    for (int64_t p = 0; p < n; ++p) {
        double x[3] = {xyzm[4 * p + 0], xyzm[4 * p + 1], xyzm[4 * p + 2]};
        double m = xyzm[4 * p + 3];
        long lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = (long)ceil(x[a] - 2.0 * h - 0.5);
            hi[a] = (long)floor(x[a] + 2.0 * h - 0.5);
            if (lo[a] < 0) lo[a] = 0;
            if (hi[a] > dims[a] - 1) hi[a] = dims[a] - 1;
        }
        for (long k = lo[2]; k <= hi[2]; ++k)
            for (long j = lo[1]; j <= hi[1]; ++j)
                for (long i = lo[0]; i <= hi[0]; ++i) {
                    double d[3] = {(double)i + 0.5 - x[0], (double)j + 0.5 - x[1],
                                   (double)k + 0.5 - x[2]};
                    double r = sqrt(dot3(d, d));
                    rho[((size_t)k * ny + j) * nx + i] += m * hho_kernel_m4(r, h);
                }
    }
}

/* ------------------------------------------------------------------------- */
/* Gladstone-Dale (Eq. 12) and the gradient by finite differences (Eq. 13)    */
/* ------------------------------------------------------------------------- */

/*
 * vol4[idx*4 + c] = {dn, gx, gy, gz} with dn = n - 1 = K rho (Eq. 12) and
 * g = grad dn = K grad rho (Eq. 13) per voxel unit. The paper says only
 * "finite differences"; the reading taken is central differences inside and
 * one-sided differences on the first and last voxel of each axis. Every axis
 * needs at least two voxels.
 */
void hho_index_field(const double* rho, int nx, int ny, int nz, double K, double* vol4) {
    int dims[3] = {nx, ny, nz};
    size_t nvox = (size_t)nx * ny * nz;
    for (size_t v = 0; v < nvox; ++v) vol4[4 * v] = K * rho[v];
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int ijk[3] = {i, j, k};
                size_t v = ((size_t)k * ny + j) * nx + i;
                for (int a = 0; a < 3; ++a) {
                    int lo[3] = {i, j, k}, hi[3] = {i, j, k};
                    double denom;
                    if (ijk[a] == 0) {
                        hi[a] = 1;
                        denom = 1.0;
                    } else if (ijk[a] == dims[a] - 1) {
                        lo[a] = dims[a] - 2;
                        denom = 1.0;
                    } else {
                        lo[a] = ijk[a] - 1;
                        hi[a] = ijk[a] + 1;
                        denom = 2.0;
                    }
                    size_t vlo = ((size_t)lo[2] * ny + lo[1]) * nx + lo[0];
                    size_t vhi = ((size_t)hi[2] * ny + hi[1]) * nx + hi[0];
                    vol4[4 * v + 1 + a] = (vol4[4 * vhi] - vol4[4 * vlo]) / denom;
                }
            }
}

/* ------------------------------------------------------------------------- */
/* Trilinear sampling of n and grad n (Sec. 3.3.1, last paragraph)            */
/* ------------------------------------------------------------------------- */

/*
 * Samples the four channels at position p with the standard 8-corner
 * trilinear formula over voxel centres. Reading: the lattice coordinate
 * u = p - 1/2 is clamped to [0, N-1] per axis (clamp to edge), the cell is
 * i0 = min(floor(u), N-2) and the weight is f = u - i0.
 */
void hho_trilinear4(const double* vol4, int nx, int ny, int nz, const double p[3], double out[4]) {
    int dims[3] = {nx, ny, nz};
    long i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double u = p[a] - 0.5;
        if (u < 0.0) u = 0.0;
        if (u > dims[a] - 1) u = dims[a] - 1;
        long c = (long)floor(u);
        if (c > dims[a] - 2) c = dims[a] - 2;
        i0[a] = c;
        f[a] = u - (double)c;
    }
    for (int c = 0; c < 4; ++c) out[c] = 0.0;
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) *
                           (dz ? f[2] : 1.0 - f[2]);
                size_t v = ((size_t)(i0[2] + dz) * ny + (i0[1] + dy)) * nx + (i0[0] + dx);
                for (int c = 0; c < 4; ++c) out[c] += w * vol4[4 * v + c];
            }
}

/* ------------------------------------------------------------------------- */
/* Refractive-index fields: the sampled grid, or an analytic field for pins   */
/* ------------------------------------------------------------------------- */

enum {
    HHO_FIELD_GRID = 0,       /* trilinear over vol4                        */
    HHO_FIELD_CONSTANT = 1,   /* dn = a                                      */
    HHO_FIELD_STRATIFIED = 2, /* dn = a + b z                                */
    HHO_FIELD_SPHERICAL = 3,  /* dn = a exp(-|p-c|^2 / (2 sigma^2))          */
    HHO_FIELD_LUNEBURG = 4    /* n = sqrt(2 - (|p-c|/R)^2) for |p-c| < R     */
};

typedef struct {
    int kind;
    int dims[3];          /* grid size (GRID only)                           */
    const double* vol4;   /* {dn, gx, gy, gz} per voxel (GRID only)          */
    double a, b, sigma, radius;
    double center[3];
} hho_field;

/* dn = n - 1 and g = grad n at p */
static void field_eval(const hho_field* F, const double p[3], double* dn, double g[3]) {
    double r[3];
    switch (F->kind) {
        case HHO_FIELD_GRID: {
            double s[4];
            hho_trilinear4(F->vol4, F->dims[0], F->dims[1], F->dims[2], p, s);
            *dn = s[0];
            g[0] = s[1];
            g[1] = s[2];
            g[2] = s[3];
            return;
        }
        case HHO_FIELD_CONSTANT:
            *dn = F->a;
            g[0] = g[1] = g[2] = 0.0;
            return;
        case HHO_FIELD_STRATIFIED:
            *dn = F->a + F->b * p[2];
            g[0] = g[1] = 0.0;
            g[2] = F->b;
            return;
        case HHO_FIELD_SPHERICAL: {
            for (int a = 0; a < 3; ++a) r[a] = p[a] - F->center[a];
            double e = F->a * exp(-dot3(r, r) / (2.0 * F->sigma * F->sigma));
            *dn = e;
            for (int a = 0; a < 3; ++a) g[a] = -e * r[a] / (F->sigma * F->sigma);
            return;
        }
        case HHO_FIELD_LUNEBURG: {
            for (int a = 0; a < 3; ++a) r[a] = p[a] - F->center[a];
            double R = F->radius;
            double s2 = dot3(r, r) / (R * R);
            if (s2 < 1.0) {
                double n = sqrt(2.0 - s2);
                *dn = n - 1.0;
                for (int a = 0; a < 3; ++a) g[a] = -r[a] / (R * R * n);
            } else {
                *dn = 0.0;
                g[0] = g[1] = g[2] = 0.0;
            }
            return;
        }
        default:
            *dn = 0.0;
            g[0] = g[1] = g[2] = 0.0;
    }
}

/* ------------------------------------------------------------------------- */
/* The march: Eqs. 14-18                                                      */
/* ------------------------------------------------------------------------- */

enum { HHO_STEP_EULER_PAPER = 0, HHO_STEP_RK4 = 1 };

typedef struct {
    int stepper;       /* HHO_STEP_EULER_PAPER (Eq. 16) or HHO_STEP_RK4       */
    int adaptive;      /* 1: Eq. 18; 0: fixed step h_fixed                    */
    double h_fixed;    /* fixed step length (voxels)                          */
    double h_min;      /* Eq. 18 lower clamp                                  */
    double h_max;      /* Eq. 18 upper clamp                                  */
    double theta_max;  /* Eq. 18 turning-angle tolerance (radians)            */
    double eps;        /* Eq. 18 regulariser (per voxel)                      */
    int max_steps;     /* steps allowed inside the box                        */
} hho_params;

/*
 * Step length. Adaptive (Eq. 18, second line, which is explicit in n and the
 * perpendicular gradient): clamp(n theta_max / (|g_perp| + eps), h_min, h_max).
 * Fixed (Sec. 4.1 "fixed-step variant"): h_fixed.
 */
static double step_length(const hho_params* P, double n, double gperp_norm) {
    if (!P->adaptive) return P->h_fixed;
    double ds = n * P->theta_max / (gperp_norm + P->eps);
    if (ds < P->h_min) ds = P->h_min;
    if (ds > P->h_max) ds = P->h_max;
    return ds;
}

/* Eq. 15 right-hand side with unnormalised w: (g - (w.g) w) / n, at C. */
static void ray_rhs(const hho_field* F, const double C[3], const double w[3], double dw[3],
                    double* n_out, double* gperp_norm_out) {
    double dn, g[3];
    field_eval(F, C, &dn, g);
    double n = 1.0 + dn;
    double wg = dot3(w, g);
    double gp[3] = {g[0] - wg * w[0], g[1] - wg * w[1], g[2] - wg * w[2]};
    for (int a = 0; a < 3; ++a) dw[a] = gp[a] / n;
    if (n_out) *n_out = n;
    if (gperp_norm_out) *gperp_norm_out = sqrt(dot3(gp, gp));
}

static int outside_box(const double C[3], const double box[3]) {
    for (int a = 0; a < 3; ++a)
        if (C[a] < 0.0 || C[a] > box[a]) return 1;
    return 0;
}

/*
 * Marches one ray from C0 (inside or on the box [0,box]) with unit direction
 * w0 and returns its exit state.
 *
 * Per step k (Sec. 3.3.2-3.3.3), at C_k with direction w_k:
 *   n_k = n(C_k), g_k = grad n(C_k), g_perp = (I - w_k w_k^T) g_k (Eq. 15),
 *   ds_k by Eq. 18 (adaptive) or fixed,
 *   EULER_PAPER (Eq. 16): w_{k+1} = normalize(w_k + ds_k/n_k g_perp),
 *                         C_{k+1} = C_k + ds_k w_{k+1};
 *   RK4 (classical four-stage RK4 of Eq. 15 in the state (C, w), w left
 *        unnormalised inside the stages, normalised at the end of the step;
 *        ds_k from the first stage).
 * Exit (reading: the paper only says rays are straight outside the volume):
 * when C_{k+1} leaves the box, the segment C_k -> C_{k+1} is clipped at the
 * box face: t* = slab exit distance from C_k along u = (C_{k+1}-C_k)/ds_k,
 * clipped to [0, ds_k]; exit position C_k + t* u, exit direction w_{k+1}.
 * After max_steps steps without leaving, the ray stops at (C, w) and the
 * MAXSTEPS flag is set.
 *
 * path (optional, path_cap rows of 7 doubles): row k = {C_k, w_k, ds_k}
 * for the steps taken (ds of the last row is the step that left, if any).
 * Returns the number of steps taken.
 */
int hho_march_ray(const hho_field* F, const double box[3], const double C0[3], const double w0[3],
                  const hho_params* P, double exit_pos[3], double exit_dir[3], int32_t* steps_out,
                  uint32_t* flags_out, double* path, int path_cap) {
    double C[3] = {C0[0], C0[1], C0[2]};
    double w[3] = {w0[0], w0[1], w0[2]};
    uint32_t flags = 0;
    int k;
    for (k = 0; k < P->max_steps; ++k) {
        double C1[3], w1[3], ds;
        if (P->stepper == HHO_STEP_RK4) {
            double k1w[3], k2w[3], k3w[3], k4w[3];
            double Cs[3], ws[3], n1, gpn1;
            ray_rhs(F, C, w, k1w, &n1, &gpn1);
            ds = step_length(P, n1, gpn1);
            for (int a = 0; a < 3; ++a) {
                Cs[a] = C[a] + 0.5 * ds * w[a];
                ws[a] = w[a] + 0.5 * ds * k1w[a];
            }
            double w2[3] = {ws[0], ws[1], ws[2]};
            ray_rhs(F, Cs, ws, k2w, NULL, NULL);
            for (int a = 0; a < 3; ++a) {
                Cs[a] = C[a] + 0.5 * ds * w2[a];
                ws[a] = w[a] + 0.5 * ds * k2w[a];
            }
            double w3[3] = {ws[0], ws[1], ws[2]};
            ray_rhs(F, Cs, ws, k3w, NULL, NULL);
            for (int a = 0; a < 3; ++a) {
                Cs[a] = C[a] + ds * w3[a];
                ws[a] = w[a] + ds * k3w[a];
            }
            double w4[3] = {ws[0], ws[1], ws[2]};
            ray_rhs(F, Cs, ws, k4w, NULL, NULL);
            for (int a = 0; a < 3; ++a) {
                C1[a] = C[a] + ds / 6.0 * (w[a] + 2.0 * w2[a] + 2.0 * w3[a] + w4[a]);
                w1[a] = w[a] + ds / 6.0 * (k1w[a] + 2.0 * k2w[a] + 2.0 * k3w[a] + k4w[a]);
            }
            normalize3(w1);
        } else {
            double dn, g[3];
            field_eval(F, C, &dn, g);
            double n = 1.0 + dn;
            double wg = dot3(w, g);
            double gp[3] = {g[0] - wg * w[0], g[1] - wg * w[1], g[2] - wg * w[2]};
            ds = step_length(P, n, sqrt(dot3(gp, gp)));
            for (int a = 0; a < 3; ++a) w1[a] = w[a] + ds / n * gp[a];
            normalize3(w1);
            for (int a = 0; a < 3; ++a) C1[a] = C[a] + ds * w1[a];
        }
        if (path && k < path_cap) {
            double* row = path + 7 * (size_t)k;
            for (int a = 0; a < 3; ++a) {
                row[a] = C[a];
                row[3 + a] = w[a];
            }
            row[6] = ds;
        }
        if (outside_box(C1, box)) {
            double u[3], tstar = INFINITY;
            for (int a = 0; a < 3; ++a) u[a] = (C1[a] - C[a]) / ds;
            for (int a = 0; a < 3; ++a) {
                double t = INFINITY;
                if (u[a] > 0.0) t = (box[a] - C[a]) / u[a];
                else if (u[a] < 0.0) t = (0.0 - C[a]) / u[a];
                if (t < tstar) tstar = t;
            }
            if (tstar < 0.0) tstar = 0.0;
            if (tstar > ds) tstar = ds;
            for (int a = 0; a < 3; ++a) {
                exit_pos[a] = C[a] + tstar * u[a];
                exit_dir[a] = w1[a];
            }
            flags |= HHO_FLAG_EXITED;
            *steps_out = k + 1;
            *flags_out = flags;
            return k + 1;
        }
        for (int a = 0; a < 3; ++a) {
            C[a] = C1[a];
            w[a] = w1[a];
        }
    }
    for (int a = 0; a < 3; ++a) {
        exit_pos[a] = C[a];
        exit_dir[a] = w[a];
    }
    flags |= HHO_FLAG_MAXSTEPS;
    *steps_out = k;
    *flags_out = flags;
    return k;
}

/* ------------------------------------------------------------------------- */
/* Ray generation and entry (rays are straight outside the volume, Fig. 1)    */
/* ------------------------------------------------------------------------- */

typedef struct {
    double eye[3], look_at[3], up[3];
    double vfov_deg;  /* vertical field of view                              */
    int width, height;
} hho_camera;

/*
 * Pinhole ray through the centre of pixel (px, py); row 0 is the top row.
 * Reading (the paper does not state its camera model): f = normalize(look_at
 * - eye), r = normalize(f x up), u = r x f, t = tan(vfov/2),
 * d = normalize(f + (2(px+1/2)/W - 1) t (W/H) r + (1 - 2(py+1/2)/H) t u).
 */
void hho_camera_ray(const hho_camera* cam, int px, int py, double dir[3]) {
    double f[3] = {cam->look_at[0] - cam->eye[0], cam->look_at[1] - cam->eye[1],
                   cam->look_at[2] - cam->eye[2]};
    normalize3(f);
    double r[3], u[3];
    cross3(f, cam->up, r);
    normalize3(r);
    cross3(r, f, u);
    double t = tan(0.5 * cam->vfov_deg * HHO_PI / 180.0);
    double W = cam->width, H = cam->height;
    double a = (2.0 * (px + 0.5) / W - 1.0) * t * (W / H);
    double b = (1.0 - 2.0 * (py + 0.5) / H) * t;
    for (int c = 0; c < 3; ++c) dir[c] = f[c] + a * r[c] + b * u[c];
    normalize3(dir);
}

/*
 * Slab test of the ray o + t d against the box [0,box]. Writes the entry and
 * exit parameters; returns 1 on a hit (t_out >= max(t_in, 0)), 0 on a miss.
 * An axis with d = 0 is a miss when o lies outside that slab.
 */
int hho_slab(const double o[3], const double d[3], const double box[3], double* t_in,
             double* t_out) {
    double tin = -INFINITY, tout = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < 0.0 || o[a] > box[a]) return 0;
            continue;
        }
        double t1 = (0.0 - o[a]) / d[a];
        double t2 = (box[a] - o[a]) / d[a];
        double tn = t1 < t2 ? t1 : t2;
        double tf = t1 < t2 ? t2 : t1;
        if (tn > tin) tin = tn;
        if (tf < tout) tout = tf;
    }
    *t_in = tin;
    *t_out = tout;
    return tout >= (tin > 0.0 ? tin : 0.0);
}

/* ------------------------------------------------------------------------- */
/* Scene radiance along the exit ray (stand-in for Sec. 3.3.2's "standard     */
/* scene intersection"): a bilinear equirectangular background               */
/* ------------------------------------------------------------------------- */

/*
 * phi = atan2(d_y, d_x), theta = atan2(sqrt(d_x^2 + d_y^2), d_z) (the polar
 * angle from +z; equal to acos(d_z) for a unit vector and well conditioned
 * near the poles). u = (phi/(2 pi) + 1/2) W - 1/2, v = (theta/pi) H - 1/2.
 * Bilinear over texel centres: u wraps, v is clamped to [0, H-1]. Texels are
 * RGB8, row-major, row 0 at theta = 0, value/255.
 */
void hho_background(const uint8_t* rgb8, int W, int H, const double d[3], double rgb[3]) {
    double phi = atan2(d[1], d[0]);
    double theta = atan2(sqrt(d[0] * d[0] + d[1] * d[1]), d[2]);
    double u = (phi / (2.0 * HHO_PI) + 0.5) * W - 0.5;
    double v = (theta / HHO_PI) * H - 0.5;
    double ifl = floor(u);
    double fu = u - ifl;
    long i0 = (long)ifl % W;
    if (i0 < 0) i0 += W;
    long i1 = (i0 + 1) % W;
    if (v < 0.0) v = 0.0;
    if (v > H - 1) v = H - 1;
    long j0 = (long)floor(v);
    if (j0 > H - 2) j0 = H - 2;
    double fv = v - (double)j0;
    long j1 = j0 + 1;
    for (int c = 0; c < 3; ++c) {
        double t00 = rgb8[((size_t)j0 * W + i0) * 3 + c] / 255.0;
        double t01 = rgb8[((size_t)j0 * W + i1) * 3 + c] / 255.0;
        double t10 = rgb8[((size_t)j1 * W + i0) * 3 + c] / 255.0;
        double t11 = rgb8[((size_t)j1 * W + i1) * 3 + c] / 255.0;
        rgb[c] = (1.0 - fv) * ((1.0 - fu) * t00 + fu * t01) + fv * ((1.0 - fu) * t10 + fu * t11);
    }
}

/*
 * Scene geometry behind the volume (the paper's scene intersection, Sec. 4.1,
 * in its simplest analytic form): textured rectangles origin + a u + b v,
 * a, b in [0, 1], u perpendicular to v; RGB8 texture row 0 at b = 0, sampled
 * bilinearly at (a W - 1/2, b H - 1/2) clamped to the texel centres. The
 * straight ray P + t d, t > 0, shows the nearest rectangle it hits, else the
 * environment map.
 */
typedef struct {
    double origin[3], u[3], v[3];
    const uint8_t* rgb8;
    int width, height;
} hho_plane;

typedef struct {
    const uint8_t* rgb8; /* environment map */
    int width, height;
    int n_planes;
    hho_plane planes[4];
} hho_scene;

static void texture_bilinear(const uint8_t* tex, int W, int H, double s, double t, double rgb[3]) {
    if (s < 0.0) s = 0.0;
    if (s > W - 1) s = W - 1;
    if (t < 0.0) t = 0.0;
    if (t > H - 1) t = H - 1;
    long i0 = (long)floor(s), j0 = (long)floor(t);
    if (i0 > W - 2) i0 = W - 2;
    if (j0 > H - 2) j0 = H - 2;
    double fs = s - (double)i0, ft = t - (double)j0;
    for (int c = 0; c < 3; ++c) {
        double t00 = tex[((size_t)j0 * W + i0) * 3 + c] / 255.0;
        double t01 = tex[((size_t)j0 * W + i0 + 1) * 3 + c] / 255.0;
        double t10 = tex[((size_t)(j0 + 1) * W + i0) * 3 + c] / 255.0;
        double t11 = tex[((size_t)(j0 + 1) * W + i0 + 1) * 3 + c] / 255.0;
        rgb[c] = (1.0 - ft) * ((1.0 - fs) * t00 + fs * t01) + ft * ((1.0 - fs) * t10 + fs * t11);
    }
}

void hho_scene_color(const hho_scene* S, const double P[3], const double d[3], double rgb[3]) {
    double best_t = INFINITY, best_a = 0.0, best_b = 0.0;
    int best = -1;
    for (int k = 0; k < S->n_planes; ++k) {
        const hho_plane* pl = &S->planes[k];
        double nrm[3], op[3], X[3], r[3];
        cross3(pl->u, pl->v, nrm);
        double den = dot3(d, nrm);
        if (den == 0.0) continue;
        for (int a = 0; a < 3; ++a) op[a] = pl->origin[a] - P[a];
        double t = dot3(op, nrm) / den;
        if (!(t > 0.0) || !(t < best_t)) continue;
        for (int a = 0; a < 3; ++a) {
            X[a] = P[a] + t * d[a];
            r[a] = X[a] - pl->origin[a];
        }
        double aa = dot3(r, pl->u) / dot3(pl->u, pl->u);
        double bb = dot3(r, pl->v) / dot3(pl->v, pl->v);
        if (aa >= 0.0 && aa <= 1.0 && bb >= 0.0 && bb <= 1.0) {
            best = k;
            best_t = t;
            best_a = aa;
            best_b = bb;
        }
    }
    if (best < 0) {
        hho_background(S->rgb8, S->width, S->height, d, rgb);
        return;
    }
    const hho_plane* pl = &S->planes[best];
    texture_bilinear(pl->rgb8, pl->width, pl->height, best_a * pl->width - 0.5,
                     best_b * pl->height - 0.5, rgb);
}

/* ------------------------------------------------------------------------- */
/* Whole pixels: ray generation -> entry -> march -> scene                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    const hho_field* F;
    double box[3];
    const hho_camera* cam;
    const hho_params* P;
    const hho_scene* scene;
    const int64_t* pixels;
    int64_t n_pix;
    double* rgb;
    double* exit_pos;
    double* exit_dir;
    int32_t* steps;
    uint32_t* flags;
    int thread, nthreads;
} trace_job;

/*
 * One pixel. A ray that misses the box keeps its straight direction: the
 * colour is the background at w0, the exit position is the eye, the exit
 * direction is w0, zero steps and no flags. A hit enters at
 * C0 = eye + max(t_in, 0) d and marches (flag HIT).
 */
static void trace_pixel(const trace_job* J, int64_t slot, int64_t pix) {
    const hho_camera* cam = J->cam;
    int px = (int)(pix % cam->width), py = (int)(pix / cam->width);
    double d[3], t_in, t_out, ep[3], ed[3];
    int32_t steps = 0;
    uint32_t flags = 0;
    hho_camera_ray(cam, px, py, d);
    if (hho_slab(cam->eye, d, J->box, &t_in, &t_out)) {
        double t0 = t_in > 0.0 ? t_in : 0.0;
        double C0[3] = {cam->eye[0] + t0 * d[0], cam->eye[1] + t0 * d[1], cam->eye[2] + t0 * d[2]};
        hho_march_ray(J->F, J->box, C0, d, J->P, ep, ed, &steps, &flags, NULL, 0);
        flags |= HHO_FLAG_HIT;
    } else {
        for (int a = 0; a < 3; ++a) {
            ep[a] = cam->eye[a];
            ed[a] = d[a];
        }
    }
    double rgb[3];
    hho_scene_color(J->scene, ep, ed, rgb);
    for (int a = 0; a < 3; ++a) {
        if (J->rgb) J->rgb[3 * slot + a] = rgb[a];
        if (J->exit_pos) J->exit_pos[3 * slot + a] = ep[a];
        if (J->exit_dir) J->exit_dir[3 * slot + a] = ed[a];
    }
    if (J->steps) J->steps[slot] = steps;
    if (J->flags) J->flags[slot] = flags;
}

static void* trace_worker(void* arg) {
    const trace_job* J = (const trace_job*)arg;
    for (int64_t s = J->thread; s < J->n_pix; s += J->nthreads)
        trace_pixel(J, s, J->pixels ? J->pixels[s] : s);
    return NULL;
}

/*
 * Traces the pixels of one camera through a field and into the scene.
 * pixels == NULL traces all
 * width*height pixels in row-major order; otherwise output slot s holds
 * pixel pixels[s] (= py*width + px). Outputs may be NULL. Work is striped
 * over nthreads POSIX threads (each pixel is independent). Returns 0.
 */
int hho_trace_field(const hho_field* F, const double box[3], const hho_camera* cam,
                    const hho_params* P, const hho_scene* scene,
                    const int64_t* pixels, int64_t n_pix, double* rgb, double* exit_pos,
                    double* exit_dir, int32_t* steps, uint32_t* flags, int nthreads) {
    if (!pixels) n_pix = (int64_t)cam->width * cam->height;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    trace_job jobs[256];
    pthread_t tid[256];
    for (int t = 0; t < nthreads; ++t) {
        trace_job* J = &jobs[t];
        J->F = F;
        for (int a = 0; a < 3; ++a) J->box[a] = box[a];
        J->cam = cam;
        J->P = P;
        J->scene = scene;
        J->pixels = pixels;
        J->n_pix = n_pix;
        J->rgb = rgb;
        J->exit_pos = exit_pos;
        J->exit_dir = exit_dir;
        J->steps = steps;
        J->flags = flags;
        J->thread = t;
        J->nthreads = nthreads;
    }
    if (nthreads == 1) {
        trace_worker(&jobs[0]);
        return 0;
    }
    for (int t = 0; t < nthreads; ++t) pthread_create(&tid[t], NULL, trace_worker, &jobs[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(tid[t], NULL);
    return 0;
}

/* Grid convenience: the box is [0,nx] x [0,ny] x [0,nz] over vol4. */
int hho_trace_grid(const double* vol4, int nx, int ny, int nz, const hho_camera* cam,
                   const hho_params* P, const hho_scene* scene,
                   const int64_t* pixels, int64_t n_pix, double* rgb, double* exit_pos,
                   double* exit_dir, int32_t* steps, uint32_t* flags, int nthreads) {
    hho_field F;
    memset(&F, 0, sizeof F);
    F.kind = HHO_FIELD_GRID;
    F.dims[0] = nx;
    F.dims[1] = ny;
    F.dims[2] = nz;
    F.vol4 = vol4;
    double box[3] = {nx, ny, nz};
    return hho_trace_field(&F, box, cam, P, scene, pixels, n_pix, rgb, exit_pos, exit_dir,
                           steps, flags, nthreads);
}

/* ------------------------------------------------------------------------- */
/* Many rays from given start states (same march, striped over threads)      */
/* ------------------------------------------------------------------------- */

typedef struct {
    const hho_field* F;
    const double* box;
    const double* C0;
    const double* w0;
    const hho_params* P;
    int64_t n;
    double* exit_pos;
    double* exit_dir;
    int32_t* steps;
    uint32_t* flags;
    int thread, nthreads;
} rays_job;

static void* rays_worker(void* arg) {
    const rays_job* J = (const rays_job*)arg;
    for (int64_t i = J->thread; i < J->n; i += J->nthreads)
        hho_march_ray(J->F, J->box, J->C0 + 3 * i, J->w0 + 3 * i, J->P, J->exit_pos + 3 * i,
                      J->exit_dir + 3 * i, J->steps + i, J->flags + i, NULL, 0);
    return NULL;
}

/* Marches n rays with start points C0[3n] and unit directions w0[3n]; the
 * results are hho_march_ray's (no HIT flag is added). Returns 0. */
int hho_march_rays(const hho_field* F, const double box[3], const double* C0, const double* w0,
                   int64_t n, const hho_params* P, double* exit_pos, double* exit_dir,
                   int32_t* steps, uint32_t* flags, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    rays_job jobs[256];
    pthread_t tid[256];
    for (int t = 0; t < nthreads; ++t) {
        rays_job J = {F, box, C0, w0, P, n, exit_pos, exit_dir, steps, flags, t, nthreads};
        jobs[t] = J;
    }
    if (nthreads == 1) {
        rays_worker(&jobs[0]);
        return 0;
    }
    for (int t = 0; t < nthreads; ++t) pthread_create(&tid[t], NULL, rays_worker, &jobs[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(tid[t], NULL);
    return 0;
}
