/*
 * apbf_oracle.c -- CPU reference (oracle) of one Adaptive Position-Based
 * Fluids step, written from the paper (Koster & Kruger, "Adaptive
 * Position-Based Fluids", IJCGA 6(3), 2016) and the textbook SPH/PBF
 * definitions it relies on. TEST INFRASTRUCTURE ONLY (see apbf_oracle.h).
 *
 * Built with -ffp-contract=off: FP32 expressions below are rounded after
 * every operation, in source order.
 *
 * Readings taken where the paper is silent:
 *  - W is poly6, grad W is spiky's gradient; the tensile term is
 *    s_corr = -k (W(r)/W(dq))^n; XSPH weights neighbours by m/rho0.
 *  - Neighbour sets are found once per step on the predicted positions
 *    (the neighbour search of Fig. 7) and kept for every iteration; pairs that separate past h
 *    contribute nothing because both kernels vanish there.
 *  - Inactive neighbours enter Eq. 7 with their last lambda (Fig. 7 computes
 *    lambda only over P_iter while Eq. 7 sums over all neighbours).
 *  - A particle of level L takes part in iterations 1..L (Eq. 9-10).
 *  - Contacts (the collision response of Fig. 7): after every position update, a predicted
 *    position strictly inside an obstacle moves to the nearest point of its
 *    surface (obstacles in order), then into the box; the prediction itself is
 *    only clamped to the box.
 *  - Pre-stabilisation (Sec. 4.3, the pre-stabilisation loop of Fig. 7) of the set of Eq. 11 for
 *    l = S, i.e. the particles of level < S: stabil_iters times, the position
 *    at the start of the step is moved out of the obstacles and into the box,
 *    and the predicted position is moved by the same amount, so v = (x* - x)/dt
 *    gains nothing from the correction.
 */
#include "apbf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the per-particle loops (the Jacobi passes, XSPH, the density
   diagnostic and the neighbour lists). Every particle's own arithmetic is the
   same at any thread count, so results are bit-identical; only whole-set
   reductions (the density statistics) and the sort stay serial. */
int orc_set_threads(int32_t nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

static const double ORC_PI = 3.14159265358979323846;

/* ---------------------------------------------------------------- kernels */

/* poly6: W(r) = 315 / (64 pi h^9) (h^2 - r^2)^3 for r < h, else 0. */
double orc_poly6(double r2, double h)
{
    double h2 = h * h;
    if (!(r2 < h2))
        return 0.0;
    double d = h2 - r2;
    return 315.0 / (64.0 * ORC_PI * pow(h, 9)) * d * d * d;
}

/* spiky: W(r) = 15 / (pi h^6) (h - r)^3 for r < h, else 0. */
double orc_spiky(double r, double h)
{
    if (!(r < h))
        return 0.0;
    double d = h - r;
    return 15.0 / (ORC_PI * pow(h, 6)) * d * d * d;
}

/* Gradient of spiky with respect to the first particle, r = x_i - x_j:
   grad W = -45 / (pi h^6) (h - |r|)^2 r / |r| for 0 < |r| < h, else 0. */
void orc_spiky_grad(const double r[3], double h, double g[3])
{
    double rl = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(rl > 0.0) || !(rl < h)) {
        g[0] = g[1] = g[2] = 0.0;
        return;
    }
    double d = h - rl;
    double c = -45.0 / (ORC_PI * pow(h, 6)) * d * d / rl;
    g[0] = c * r[0];
    g[1] = c * r[1];
    g[2] = c * r[2];
}

/* Eq. 6 at a particle of an infinite jitter-free cubic lattice, self term included. */
double orc_rest_density(double h, double mass, double spacing)
{
    if (!(h > 0.0) || !(spacing > 0.0))
        return -1.0;
    int k = (int)ceil(h / spacing) + 1;
    double rho = 0.0;
    for (int a = -k; a <= k; ++a)
        for (int b = -k; b <= k; ++b)
            for (int c = -k; c <= k; ++c) {
                double r2 = ((double)a * a + (double)b * b + (double)c * c) * spacing * spacing;
                rho += mass * orc_poly6(r2, h);
            }
    return rho;
}

/* ------------------------------------------------------ FP32 decisions */

int orc_grid_dims(const orc_params *p, int32_t dims[3])
{
    if (!p || !(p->h > 0.0f))
        return -1;
    float inv_h = 1.0f / p->h;
    for (int a = 0; a < 3; ++a) {
        float ext = p->grid_hi[a] - p->grid_lo[a];
        if (!(ext >= 0.0f))
            return -1;
        float t = ext * inv_h;
        dims[a] = (int32_t)floorf(t) + 1;
    }
    return 0;
}

/* Distance to camera (Sec. 4.1), linear interpolation between the distance
   range and the level range (Sec. 4.1): near -> n_max, far -> n_min, with
   K = n_max - n_min + 1 bins of equal width over the range. */

/* ---------------------------------------------------------------- DTVS */

static float dot3(const float a[3], const float b[3])
{
    float s = a[0] * b[0] + a[1] * b[1];
    s = s + a[2] * b[2];
    return s;
}

static int normalize3(float v[3])
{
    float n = sqrtf(dot3(v, v));
    if (!(n > 0.0f))
        return -1;
    v[0] = v[0] / n;
    v[1] = v[1] / n;
    v[2] = v[2] / n;
    return 0;
}

static void cross3(const float a[3], const float b[3], float c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static float depth_empty(void)
{
    uint32_t u = 0x7f7f7f7fu;
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
}

int orc_view_basis(const orc_view *v, float f[3], float r[3], float u[3])
{
    if (!v)
        return -1;
    for (int a = 0; a < 3; ++a)
        f[a] = v->dir[a];
    if (normalize3(f))
        return -1;
    cross3(f, v->up, r);
    if (normalize3(r))
        return -1;
    cross3(r, f, u);
    return 0;
}

/* The image plane at unit distance spans [-ax, ax] x [-ay, ay]. */
static void half_extents(const orc_view *v, float *ax, float *ay)
{
    *ax = v->tan_half_fov * ((float)v->width / (float)v->height);
    *ay = v->tan_half_fov;
}

int orc_pixel_ray(const orc_view *v, int32_t px, int32_t py, float ray[3])
{
    float f[3], r[3], u[3], ax, ay;
    if (orc_view_basis(v, f, r, u))
        return -1;
    half_extents(v, &ax, &ay);
    float sx = ((float)(2 * px + 1) / (float)v->width - 1.0f) * ax;
    float sy = (1.0f - (float)(2 * py + 1) / (float)v->height) * ay;
    for (int a = 0; a < 3; ++a) {
        float c = f[a] + sx * r[a];
        ray[a] = c + sy * u[a];
    }
    return normalize3(ray);
}

static int view_ok(const orc_view *v)
{
    return v->width >= 1 && v->height >= 1 && v->tan_half_fov > 0.0f && v->radius > 0.0f;
}

int orc_depth_image(const orc_params *p, int32_t n, const float *x, float *depth)
{
    if (!p || n < 0 || (n > 0 && !x) || !depth || !view_ok(&p->view))
        return -1;
    const orc_view *v = &p->view;
    const int32_t W = v->width, H = v->height;
    float f[3], r[3], u[3], ax, ay;
    if (orc_view_basis(v, f, r, u))
        return -1;
    half_extents(v, &ax, &ay);
    float *rays = (float *)malloc(sizeof(float) * 3 * (size_t)W * (size_t)H);
    if (!rays)
        return -3;
    for (int32_t py = 0; py < H; ++py)
        for (int32_t px = 0; px < W; ++px) {
            orc_pixel_ray(v, px, py, rays + 3 * ((size_t)py * W + px));
            depth[(size_t)py * W + px] = depth_empty();
        }
    const float r2 = v->radius * v->radius;
    for (int32_t i = 0; i < n; ++i) {
        float rel[3] = {x[3 * i + 0] - p->eye[0], x[3 * i + 1] - p->eye[1], x[3 * i + 2] - p->eye[2]};
        float cc = dot3(rel, rel) - r2;
        if (!(cc > 0.0f))
            continue; /* the eye is inside this sphere: it is not rendered */
        /* pixels to test: all, or a box around the projections of the 8
           corners of the sphere's bounding cube, widened by one pixel (a
           conservative cull that does not change the image) */
        int32_t x0 = 0, x1 = W - 1, y0 = 0, y1 = H - 1;
        if (!v->brute_force) {
            float fx_lo = INFINITY, fx_hi = -INFINITY, fy_lo = INFINITY, fy_hi = -INFINITY;
            int behind = 0;
            for (int c = 0; c < 8; ++c) {
                float q[3] = {rel[0] + ((c & 1) ? v->radius : -v->radius), rel[1] + ((c & 2) ? v->radius : -v->radius),
                              rel[2] + ((c & 4) ? v->radius : -v->radius)};
                float zc = dot3(q, f);
                if (!(zc > 0.0f)) {
                    behind = 1;
                    break;
                }
                float fx = ((dot3(q, r) / zc) / ax + 1.0f) * (0.5f * (float)W);
                float fy = (1.0f - (dot3(q, u) / zc) / ay) * (0.5f * (float)H);
                fx_lo = fminf(fx_lo, fx);
                fx_hi = fmaxf(fx_hi, fx);
                fy_lo = fminf(fy_lo, fy);
                fy_hi = fmaxf(fy_hi, fy);
            }
            if (!behind) {
                if (fx_hi < -1.0f || fy_hi < -1.0f || fx_lo > (float)W + 1.0f || fy_lo > (float)H + 1.0f)
                    continue; /* entirely outside the image */
                x0 = (int32_t)floorf(fmaxf(fx_lo, -1.0f)) - 1;
                x1 = (int32_t)floorf(fminf(fx_hi, (float)W + 1.0f)) + 1;
                y0 = (int32_t)floorf(fmaxf(fy_lo, -1.0f)) - 1;
                y1 = (int32_t)floorf(fminf(fy_hi, (float)H + 1.0f)) + 1;
                x0 = x0 < 0 ? 0 : x0;
                y0 = y0 < 0 ? 0 : y0;
                x1 = x1 > W - 1 ? W - 1 : x1;
                y1 = y1 > H - 1 ? H - 1 : y1;
            }
        }
        for (int32_t py = y0; py <= y1; ++py)
            for (int32_t px = x0; px <= x1; ++px) {
                const float *ray = rays + 3 * ((size_t)py * W + px);
                float b = dot3(ray, rel); /* distance along the ray to the centre's foot point */
                if (!(b > 0.0f))
                    continue;
                /* squared half chord r^2 - |rel - b ray|^2: the perpendicular
                   offset is formed first, which keeps the difference well conditioned */
                float w[3] = {rel[0] - b * ray[0], rel[1] - b * ray[1], rel[2] - b * ray[2]};
                float disc = r2 - dot3(w, w);
                if (!(disc >= 0.0f))
                    continue;
                float t = b - sqrtf(disc);
                if (!(t > 0.0f))
                    continue; /* the image holds distances in front of the camera */
                float *dp = depth + (size_t)py * W + px;
                if (t < *dp)
                    *dp = t;
            }
    }
    free(rays);
    return 0;
}

int orc_dtvs_distance(const orc_params *p, int32_t n, const float *x, const float *depth, float *dist)
{
    if (!p || n < 0 || (n > 0 && (!x || !dist)) || !depth || !view_ok(&p->view))
        return -1;
    const orc_view *v = &p->view;
    float f[3], r[3], u[3], ax, ay;
    if (orc_view_basis(v, f, r, u))
        return -1;
    half_extents(v, &ax, &ay);
    for (int32_t i = 0; i < n; ++i) {
        float rel[3] = {x[3 * i + 0] - p->eye[0], x[3 * i + 1] - p->eye[1], x[3 * i + 2] - p->eye[2]};
        float zc = dot3(rel, f);
        dist[i] = -1.0f;
        if (!(zc > 0.0f))
            continue;
        float fx = ((dot3(rel, r) / zc) / ax + 1.0f) * (0.5f * (float)v->width);
        float fy = (1.0f - (dot3(rel, u) / zc) / ay) * (0.5f * (float)v->height);
        if (!(fx >= 0.0f && fx < (float)v->width && fy >= 0.0f && fy < (float)v->height))
            continue;
        int32_t px = (int32_t)floorf(fx), py = (int32_t)floorf(fy);
        float front = sqrtf(dot3(rel, rel)) - v->radius;
        float d = front - depth[(size_t)py * v->width + px];
        dist[i] = d > 0.0f ? d : 0.0f;
    }
    return 0;
}

int orc_lod_levels(const orc_params *p, int32_t n, const float *x, int32_t *level, float range[2])
{
    if (!p || n < 0 || (n > 0 && (!x || !level)))
        return -1;
    if (p->n_min < 1 || p->n_max < p->n_min)
        return -1;
    if (p->lod_mode == ORC_LOD_FIXED) {
        for (int32_t i = 0; i < n; ++i)
            level[i] = p->n_max;
        if (range) {
            range[0] = 0.0f;
            range[1] = 0.0f;
        }
        return 0;
    }
    if (p->lod_mode != ORC_LOD_DTC && p->lod_mode != ORC_LOD_DTVS)
        return -1;
    if (p->lod_mode == ORC_LOD_DTVS && p->view.outside_level != 0 &&
        (p->view.outside_level < p->n_min || p->view.outside_level > p->n_max))
        return -1;
    float *d = (float *)malloc(sizeof(float) * (size_t)(n > 0 ? n : 1));
    if (!d)
        return -3;
    if (p->lod_mode == ORC_LOD_DTC) {
        for (int32_t i = 0; i < n; ++i) {
            float dx = x[3 * i + 0] - p->eye[0];
            float dy = x[3 * i + 1] - p->eye[1];
            float dz = x[3 * i + 2] - p->eye[2];
            float d2 = dx * dx + dy * dy;
            d2 = d2 + dz * dz;
            d[i] = sqrtf(d2);
        }
    } else {
        if (!view_ok(&p->view)) {
            free(d);
            return -1;
        }
        float *depth = (float *)malloc(sizeof(float) * (size_t)p->view.width * (size_t)p->view.height);
        if (!depth) {
            free(d);
            return -3;
        }
        int rc = orc_depth_image(p, n, x, depth);
        if (rc == 0)
            rc = orc_dtvs_distance(p, n, x, depth, d);
        free(depth);
        if (rc) {
            free(d);
            return rc;
        }
    }
    int automatic = !(p->d_near < p->d_far);
    float dmin = p->d_near, dmax = p->d_far;
    if (automatic) {
        int32_t seen = 0;
        dmin = INFINITY;
        dmax = 0.0f;
        for (int32_t i = 0; i < n; ++i) {
            if (d[i] < 0.0f)
                continue; /* DTVS: outside the view */
            ++seen;
            if (d[i] < dmin)
                dmin = d[i];
            if (d[i] > dmax)
                dmax = d[i];
        }
        if (seen == 0)
            dmin = dmax = 0.0f;
    }
    int32_t K = p->n_max - p->n_min + 1;
    float span = dmax - dmin;
    for (int32_t i = 0; i < n; ++i) {
        if (d[i] < 0.0f) { /* DTVS: outside the view */
            level[i] = p->view.outside_level ? p->view.outside_level : p->n_min;
            continue;
        }
        float t = 0.0f;
        if (span > 0.0f) {
            float num = d[i] - dmin;
            t = num / span;
        }
        if (t < 0.0f)
            t = 0.0f;
        if (t > 1.0f)
            t = 1.0f;
        if (p->lod_rounding == 0) {
            float tk = t * (float)K;
            int32_t b = (int32_t)floorf(tk);
            if (b > K - 1)
                b = K - 1;
            level[i] = p->n_max - b;
        } else {
            double lv = (double)p->n_max + (double)t * ((double)p->n_min - (double)p->n_max);
            level[i] = (int32_t)floor(lv + 0.5);
        }
    }
    if (range) {
        range[0] = dmin;
        range[1] = dmax;
    }
    free(d);
    return 0;
}

/* The prediction step of Fig. 7: v' = v + dt g, x* = x + dt v', then x* clamped to the box. */
int orc_predict(const orc_params *p, int32_t n, const float *x, const float *v, float *xpred)
{
    if (!p || n < 0 || (n > 0 && (!x || !v || !xpred)))
        return -1;
    for (int32_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            float vv = v[3 * i + a] + p->dt * p->gravity[a];
            float xp = x[3 * i + a] + p->dt * vv;
            xp = fmaxf(xp, p->box_lo[a]);
            xp = fminf(xp, p->box_hi[a]);
            xpred[3 * i + a] = xp;
        }
    return 0;
}

static void cell_coords(const orc_params *p, const int32_t dims[3], float inv_h, const float *xq,
                        int32_t c[3])
{
    for (int a = 0; a < 3; ++a) {
        float rel = xq[a] - p->grid_lo[a];
        float t = rel * inv_h;
        int32_t k = (int32_t)floorf(t);
        if (k < 0)
            k = 0;
        if (k > dims[a] - 1)
            k = dims[a] - 1;
        c[a] = k;
    }
}

/* key = (cz * ny + cy) * nx + cx on the uniform grid of cell size h. */
int orc_cell_keys(const orc_params *p, int32_t n, const float *xpos, uint32_t *keys)
{
    int32_t dims[3];
    if (orc_grid_dims(p, dims) != 0 || n < 0 || (n > 0 && (!xpos || !keys)))
        return -1;
    float inv_h = 1.0f / p->h;
    for (int32_t i = 0; i < n; ++i) {
        int32_t c[3];
        cell_coords(p, dims, inv_h, xpos + 3 * i, c);
        keys[i] = (uint32_t)(((int64_t)c[2] * dims[1] + c[1]) * dims[0] + c[0]);
    }
    return 0;
}

/* Textbook counting sort: histogram, exclusive prefix sum, then a pass in
   input order that places each element after the earlier ones of its key. */
int orc_counting_sort(int32_t n, const uint32_t *keys, int64_t ncell, int32_t *order, uint32_t *cell_start)
{
    if (n < 0 || ncell < 1 || (n > 0 && (!keys || !order)) || !cell_start)
        return -1;
    uint32_t *fill = (uint32_t *)calloc((size_t)ncell, sizeof(uint32_t));
    if (!fill)
        return -3;
    memset(cell_start, 0, sizeof(uint32_t) * (size_t)(ncell + 1));
    for (int32_t i = 0; i < n; ++i) {
        if ((int64_t)keys[i] >= ncell) {
            free(fill);
            return -1;
        }
        cell_start[keys[i] + 1] += 1;
    }
    for (int64_t c = 0; c < ncell; ++c)
        cell_start[c + 1] += cell_start[c];
    for (int32_t i = 0; i < n; ++i) {
        uint32_t k = keys[i];
        order[cell_start[k] + fill[k]] = i;
        fill[k] += 1;
    }
    free(fill);
    return 0;
}

/* FP32 neighbour predicate: dx = x_i - x_j per axis, r2 = (dx^2 + dy^2) + dz^2,
   neighbour iff r2 < h*h (all FP32). */
static int is_neighbor(const float *xi, const float *xj, float h2)
{
    float dx = xi[0] - xj[0];
    float dy = xi[1] - xj[1];
    float dz = xi[2] - xj[2];
    float r2 = dx * dx + dy * dy;
    r2 = r2 + dz * dz;
    return r2 < h2;
}

/* Neighbour sets of particles already in counting-sort order (xs32 sorted,
   cell_start from the sort). Two passes: count then fill. */
static int build_neighbors_sorted(const orc_params *p, const int32_t dims[3], int32_t n,
                                  const float *xs32, const uint32_t *cell_start, int32_t **off_out,
                                  int32_t **idx_out)
{
    float inv_h = 1.0f / p->h;
    float h2 = p->h * p->h;
    int32_t *off = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    if (!off)
        return -3;
    int32_t *idx = NULL;
    for (int pass = 0; pass < 2; ++pass) {
        /* pass 0 counts each list into off[i + 1], pass 1 fills it from off[i] */
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < n; ++i) {
            int32_t c[3];
            cell_coords(p, dims, inv_h, xs32 + 3 * i, c);
            int64_t w = pass == 0 ? 0 : off[i];
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int32_t cx = c[0] + dx, cy = c[1] + dy, cz = c[2] + dz;
                        if (cx < 0 || cy < 0 || cz < 0 || cx >= dims[0] || cy >= dims[1] || cz >= dims[2])
                            continue;
                        int64_t key = ((int64_t)cz * dims[1] + cy) * dims[0] + cx;
                        for (uint32_t j = cell_start[key]; j < cell_start[key + 1]; ++j) {
                            if ((int32_t)j == i)
                                continue;
                            if (is_neighbor(xs32 + 3 * i, xs32 + 3 * j, h2)) {
                                if (pass == 1)
                                    idx[w] = (int32_t)j;
                                ++w;
                            }
                        }
                    }
            if (pass == 0)
                off[i + 1] = (int32_t)w;
        }
        if (pass == 0) {
            int64_t total = 0;
            off[0] = 0;
            for (int32_t i = 0; i < n; ++i) {
                total += off[i + 1];
                off[i + 1] = (int32_t)total;
            }
            idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
            if (!idx) {
                free(off);
                return -3;
            }
        }
    }
    /* each list ascending (cells are visited in key order, slots ascending within a cell) */
    *off_out = off;
    *idx_out = idx;
    return 0;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Neighbour sets in input indices, each list ascending; CSR arrays are
   allocated here and returned to the caller. */
static int neighbors_alloc(const orc_params *p, int32_t n, const float *x, int32_t **off_out,
                           int32_t **idx_out)
{
    int32_t dims[3];
    if (orc_grid_dims(p, dims) != 0 || n < 0 || (n > 0 && !x))
        return -1;
    int64_t ncell = (int64_t)dims[0] * dims[1] * dims[2];
    size_t nn = (size_t)(n > 0 ? n : 1);
    uint32_t *keys = (uint32_t *)malloc(sizeof(uint32_t) * nn);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * nn);
    uint32_t *start = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(ncell + 1));
    float *xs = (float *)malloc(sizeof(float) * 3 * nn);
    int32_t *deg = (int32_t *)calloc(nn, sizeof(int32_t));
    int32_t *off = (int32_t *)malloc(sizeof(int32_t) * (nn + 1));
    int32_t *soff = NULL, *sidx = NULL, *idx = NULL;
    int rc = -3;
    if (!keys || !order || !start || !xs || !deg || !off)
        goto done;
    orc_cell_keys(p, n, x, keys);
    rc = orc_counting_sort(n, keys, ncell, order, start);
    if (rc)
        goto done;
    for (int32_t s = 0; s < n; ++s)
        memcpy(xs + 3 * s, x + 3 * order[s], 3 * sizeof(float));
    rc = build_neighbors_sorted(p, dims, n, xs, start, &soff, &sidx);
    if (rc)
        goto done;
    rc = -3;
    idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(soff[n] > 0 ? soff[n] : 1));
    if (!idx)
        goto done;
    /* slot s holds input particle order[s] */
    for (int32_t s = 0; s < n; ++s)
        deg[order[s]] = soff[s + 1] - soff[s];
    off[0] = 0;
    for (int32_t i = 0; i < n; ++i)
        off[i + 1] = off[i] + deg[i];
#pragma omp parallel for schedule(static)
    for (int32_t s = 0; s < n; ++s) {
        int32_t i = order[s];
        int32_t w = off[i];
        for (int32_t k = soff[s]; k < soff[s + 1]; ++k)
            idx[w++] = order[sidx[k]];
        qsort(idx + off[i], (size_t)(off[i + 1] - off[i]), sizeof(int32_t), cmp_i32);
    }
    *off_out = off;
    *idx_out = idx;
    off = NULL;
    idx = NULL;
    rc = 0;
done:
    free(keys);
    free(order);
    free(start);
    free(xs);
    free(deg);
    free(off);
    free(idx);
    free(soff);
    free(sidx);
    return rc;
}

int orc_neighbors(const orc_params *p, int32_t n, const float *x, int32_t *off, int32_t *idx, int64_t cap)
{
    if (!off)
        return -1;
    int32_t *o = NULL, *ix = NULL;
    int rc = neighbors_alloc(p, n, x, &o, &ix);
    if (rc)
        return rc;
    if (o[n] > cap || (o[n] > 0 && !idx)) {
        off[n] = o[n];
        free(o);
        free(ix);
        return -2;
    }
    memcpy(off, o, sizeof(int32_t) * (size_t)(n + 1));
    if (o[n] > 0)
        memcpy(idx, ix, sizeof(int32_t) * (size_t)o[n]);
    free(o);
    free(ix);
    return 0;
}

/* ------------------------------------------------------- FP64 solver */

static void sub3(const double *a, const double *b, double r[3])
{
    r[0] = a[0] - b[0];
    r[1] = a[1] - b[1];
    r[2] = a[2] - b[2];
}

/* Eq. 5-6 and Eq. 4 for one particle. With uniform mass m and w = 1/m:
   rho_i = m (W(0) + sum_j W_ij),  C_i = rho_i / rho0 - 1,
   dC_i/dx_i = (m/rho0) sum_j gradW_ij,  dC_i/dx_j = -(m/rho0) gradW_ij,
   lambda_i = -C_i / (w sum_k |dC_i/dx_k|^2 + eps). */
int orc_constraint(const orc_params *p, int32_t n, const double *xs, const int32_t *nbr_off,
                   const int32_t *nbr_idx, int32_t i, double *rho_out, double *C_out, double *grad,
                   double *lambda_out)
{
    if (!p || i < 0 || i >= n || !xs || !nbr_off)
        return -1;
    double h = p->h, m = p->mass, rho0 = p->rho0, w = 1.0 / (double)p->mass;
    double rho = m * orc_poly6(0.0, h);
    double gi[3] = {0.0, 0.0, 0.0};
    double sum_sq = 0.0;
    int32_t k0 = nbr_off[i], k1 = nbr_off[i + 1];
    for (int32_t k = k0; k < k1; ++k) {
        int32_t j = nbr_idx[k];
        double r[3], g[3];
        sub3(xs + 3 * i, xs + 3 * j, r);
        rho += m * orc_poly6(r[0] * r[0] + r[1] * r[1] + r[2] * r[2], h);
        orc_spiky_grad(r, h, g);
        double gj[3] = {-(m / rho0) * g[0], -(m / rho0) * g[1], -(m / rho0) * g[2]};
        gi[0] -= gj[0];
        gi[1] -= gj[1];
        gi[2] -= gj[2];
        sum_sq += gj[0] * gj[0] + gj[1] * gj[1] + gj[2] * gj[2];
        if (grad) {
            grad[3 * (k - k0 + 1) + 0] = gj[0];
            grad[3 * (k - k0 + 1) + 1] = gj[1];
            grad[3 * (k - k0 + 1) + 2] = gj[2];
        }
    }
    sum_sq += gi[0] * gi[0] + gi[1] * gi[1] + gi[2] * gi[2];
    if (grad) {
        grad[0] = gi[0];
        grad[1] = gi[1];
        grad[2] = gi[2];
    }
    double C = rho / rho0 - 1.0;
    double lam = -C / (w * sum_sq + (double)p->eps);
    if (rho_out)
        *rho_out = rho;
    if (C_out)
        *C_out = C;
    if (lambda_out)
        *lambda_out = lam;
    return 0;
}

/* s_corr = -k (W(r) / W(dq))^n, the tensile term added to lambda_i + lambda_j. */
static double scorr(const orc_params *p, double r2)
{
    double wq = orc_poly6((double)p->scorr_dq * (double)p->scorr_dq, p->h);
    if (!(wq > 0.0) || p->scorr_k == 0.0f)
        return 0.0;
    double ratio = orc_poly6(r2, p->h) / wq;
    double pw = 1.0;
    for (int32_t e = 0; e < p->scorr_n; ++e)
        pw *= ratio;
    return -(double)p->scorr_k * pw;
}

/* Eq. 7 with the tensile term, derived from Eq. 3 summed over the density
   constraints: dp_i = (w m / rho0) sum_j (lambda_i + lambda_j + s_corr_ij) gradW_ij
   (w m = 1 for uniform mass). */
static void delta_p_one(const orc_params *p, const double *xs, const double *lam, const int32_t *nbr_off,
                        const int32_t *nbr_idx, int32_t i, double dp[3])
{
    double h = p->h, wm = (1.0 / (double)p->mass) * (double)p->mass, rho0 = p->rho0;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int32_t k = nbr_off[i]; k < nbr_off[i + 1]; ++k) {
        int32_t j = nbr_idx[k];
        double r[3], g[3];
        sub3(xs + 3 * i, xs + 3 * j, r);
        orc_spiky_grad(r, h, g);
        double s = lam[i] + lam[j] + scorr(p, r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        acc[0] += s * g[0];
        acc[1] += s * g[1];
        acc[2] += s * g[2];
    }
    dp[0] = wm / rho0 * acc[0];
    dp[1] = wm / rho0 * acc[1];
    dp[2] = wm / rho0 * acc[2];
}

int orc_delta_p(const orc_params *p, int32_t n, const double *xs, const double *lam,
                const int32_t *nbr_off, const int32_t *nbr_idx, double *dp)
{
    if (!p || n < 0 || (n > 0 && (!xs || !lam || !nbr_off || !dp)))
        return -1;
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i)
        delta_p_one(p, xs, lam, nbr_off, nbr_idx, i, dp + 3 * i);
    return 0;
}

/* XSPH: v_i += c sum_j (m / rho0) (v_j - v_i) W(x_i - x_j), from the
   velocities before smoothing (Jacobi). */
int orc_xsph(const orc_params *p, int32_t n, const double *xs, const double *v, const int32_t *nbr_off,
             const int32_t *nbr_idx, double *vout)
{
    if (!p || n < 0 || (n > 0 && (!xs || !v || !nbr_off || !vout)))
        return -1;
    double c = p->xsph_c, mr = (double)p->mass / (double)p->rho0;
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int32_t k = nbr_off[i]; k < nbr_off[i + 1]; ++k) {
            int32_t j = nbr_idx[k];
            double r[3];
            sub3(xs + 3 * i, xs + 3 * j, r);
            double W = orc_poly6(r[0] * r[0] + r[1] * r[1] + r[2] * r[2], p->h);
            for (int a = 0; a < 3; ++a)
                acc[a] += mr * (v[3 * j + a] - v[3 * i + a]) * W;
        }
        for (int a = 0; a < 3; ++a)
            vout[3 * i + a] = v[3 * i + a] + c * acc[a];
    }
    return 0;
}

int orc_obstacle_project(const orc_obstacle *o, const double x[3], double q[3])
{
    q[0] = x[0];
    q[1] = x[1];
    q[2] = x[2];
    if (!o)
        return 0;
    if (o->kind == ORC_OBSTACLE_SPHERE) {
        double d[3] = {x[0] - o->a[0], x[1] - o->a[1], x[2] - o->a[2]};
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]), R = o->b[0];
        if (!(r < R))
            return 0;
        if (r == 0.0) {
            q[2] = o->a[2] + R;
            return 1;
        }
        for (int k = 0; k < 3; ++k)
            q[k] = o->a[k] + R * d[k] / r;
        return 1;
    }
    if (o->kind == ORC_OBSTACLE_BOX) {
        double best = INFINITY, face = 0.0;
        int axis = -1;
        for (int k = 0; k < 3; ++k) {
            if (!(x[k] > o->a[k] && x[k] < o->b[k]))
                return 0;
            double dl = x[k] - o->a[k], dh = o->b[k] - x[k];
            if (dl < best) {
                best = dl;
                axis = k;
                face = o->a[k];
            }
            if (dh < best) {
                best = dh;
                axis = k;
                face = o->b[k];
            }
        }
        q[axis] = face;
        return 1;
    }
    if (o->kind == ORC_OBSTACLE_CONE) {
        /* in the half plane (rho, z) through the axis the solid is the right
           triangle (0, zb), (R, zb), (0, zb + H) */
        const double R = o->b[0], H = o->b[1], zb = o->a[2];
        double ux = x[0] - o->a[0], uy = x[1] - o->a[1];
        double rho = sqrt(ux * ux + uy * uy), z = x[2] - zb;
        if (!(z > 0.0 && rho / R + z / H < 1.0))
            return 0;
        double L = sqrt(R * R + H * H);
        double g = (H * rho + R * z - R * H) / L; /* signed distance to the slant line, < 0 inside */
        if (z <= -g) {
            q[2] = zb; /* the base is nearest */
            return 1;
        }
        double rho2 = rho - g * H / L, z2 = z - g * R / L;
        if (rho > 0.0) {
            ux /= rho;
            uy /= rho;
        } else {
            ux = 1.0;
            uy = 0.0;
        }
        q[0] = o->a[0] + rho2 * ux;
        q[1] = o->a[1] + rho2 * uy;
        q[2] = zb + z2;
        return 1;
    }
    return 0;
}

static void contact_obstacles(const orc_params *p, double *x3)
{
    for (int32_t k = 0; k < p->n_obstacles; ++k) {
        double q[3];
        if (orc_obstacle_project(&p->obstacles[k], x3, q)) {
            x3[0] = q[0];
            x3[1] = q[1];
            x3[2] = q[2];
        }
    }
}

static void clamp_box(const orc_params *p, double *x3)
{
    for (int a = 0; a < 3; ++a) {
        if (x3[a] < (double)p->box_lo[a])
            x3[a] = (double)p->box_lo[a];
        if (x3[a] > (double)p->box_hi[a])
            x3[a] = (double)p->box_hi[a];
    }
}

static int validate(const orc_params *p, int32_t n)
{
    if (!p || n < 0)
        return -1;
    if (!(p->h > 0.0f) || !(p->dt > 0.0f) || !(p->mass > 0.0f) || !(p->rho0 > 0.0f) || !(p->eps >= 0.0f))
        return -1;
    if (p->n_min < 1 || p->n_max < p->n_min || p->scorr_n < 0)
        return -1;
    if (p->n_obstacles < 0 || p->n_obstacles > ORC_MAX_OBSTACLES || p->stabil_iters < 0 || p->stabil_s < 0)
        return -1;
    for (int a = 0; a < 3; ++a)
        if (!(p->grid_lo[a] <= p->box_lo[a]) || !(p->box_lo[a] < p->box_hi[a]) ||
            !(p->box_hi[a] <= p->grid_hi[a]))
            return -1;
    return 0;
}

/* One step of Fig. 7. */
int orc_step(const orc_params *p, int32_t n, float *x, float *v, int32_t *id, orc_record *rec)
{
    if (validate(p, n) != 0 || (n > 0 && (!x || !v || !id)))
        return -1;
    int32_t dims[3];
    orc_grid_dims(p, dims);
    int64_t ncell = (int64_t)dims[0] * dims[1] * dims[2];
    size_t nn = (size_t)(n > 0 ? n : 1);
    int rc = -3;

    int32_t *level0 = (int32_t *)malloc(sizeof(int32_t) * nn);
    float *xpred = (float *)malloc(sizeof(float) * 3 * nn);
    uint32_t *keys = (uint32_t *)malloc(sizeof(uint32_t) * nn);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * nn);
    uint32_t *start = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(ncell + 1));
    float *xs32 = (float *)malloc(sizeof(float) * 3 * nn);
    float *x0s = (float *)malloc(sizeof(float) * 3 * nn);
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *lvl = (int32_t *)malloc(sizeof(int32_t) * nn);
    double *xs = (double *)malloc(sizeof(double) * 3 * nn);
    double *dp = (double *)malloc(sizeof(double) * 3 * nn);
    double *lam = (double *)calloc(nn, sizeof(double));
    double *vel = (double *)malloc(sizeof(double) * 3 * nn);
    double *vout = (double *)malloc(sizeof(double) * 3 * nn);
    double *x0d = (double *)malloc(sizeof(double) * 3 * nn);
    int32_t *noff = NULL, *nidx = NULL;
    if (!level0 || !xpred || !keys || !order || !start || !xs32 || !x0s || !ids || !lvl || !xs || !dp ||
        !lam || !vel || !vout || !x0d)
        goto done;

    /* LOD from the positions at the start of the step (Sec. 4.1, Sec. 6). */
    float range[2] = {0.0f, 0.0f};
    rc = orc_lod_levels(p, n, x, level0, range);
    if (rc)
        goto done;
    /* The prediction step of Fig. 7 (FP32). */
    orc_predict(p, n, x, v, xpred);
    /* The neighbour search of Fig. 7: counting sort by cell, ties by particle id (the
       counting sort is stable and is fed the particles in id order), then
       neighbour sets. */
    orc_cell_keys(p, n, xpred, keys);
    {
        int32_t *pos_of_id = (int32_t *)malloc(sizeof(int32_t) * nn);
        uint32_t *keys_by_id = (uint32_t *)malloc(sizeof(uint32_t) * nn);
        if (!pos_of_id || !keys_by_id) {
            free(pos_of_id);
            free(keys_by_id);
            rc = -3;
            goto done;
        }
        rc = 0;
        for (int32_t i = 0; i < n; ++i) {
            if (id[i] < 0 || id[i] >= n)
                rc = -1;
            else
                pos_of_id[id[i]] = i;
        }
        if (rc == 0) {
            for (int32_t k = 0; k < n; ++k)
                keys_by_id[k] = keys[pos_of_id[k]];
            rc = orc_counting_sort(n, keys_by_id, ncell, order, start);
            for (int32_t s = 0; s < n && rc == 0; ++s)
                order[s] = pos_of_id[order[s]];
        }
        free(pos_of_id);
        free(keys_by_id);
        if (rc)
            goto done;
    }
    for (int32_t s = 0; s < n; ++s) {
        int32_t i = order[s];
        memcpy(xs32 + 3 * s, xpred + 3 * i, 3 * sizeof(float));
        memcpy(x0s + 3 * s, x + 3 * i, 3 * sizeof(float));
        ids[s] = id[i];
        lvl[s] = level0[i];
    }
    rc = build_neighbors_sorted(p, dims, n, xs32, start, &noff, &nidx);
    if (rc)
        goto done;

    if (rec) {
        if (rec->xpred)
            memcpy(rec->xpred, xpred, sizeof(float) * 3 * (size_t)n);
        if (rec->level_presort)
            memcpy(rec->level_presort, level0, sizeof(int32_t) * (size_t)n);
        if (rec->keys)
            memcpy(rec->keys, keys, sizeof(uint32_t) * (size_t)n);
        if (rec->order)
            memcpy(rec->order, order, sizeof(int32_t) * (size_t)n);
        if (rec->cell_start) {
            if (rec->cell_cap < ncell + 1) {
                rc = -2;
                goto done;
            }
            memcpy(rec->cell_start, start, sizeof(uint32_t) * (size_t)(ncell + 1));
        }
        if (rec->nbr_off)
            memcpy(rec->nbr_off, noff, sizeof(int32_t) * (size_t)(n + 1));
        if (rec->nbr_idx) {
            if (rec->nbr_cap < noff[n]) {
                rc = -2;
                goto done;
            }
            memcpy(rec->nbr_idx, nidx, sizeof(int32_t) * (size_t)noff[n]);
        }
        if (rec->active_count)
            for (int32_t l = 0; l <= p->n_max + 1; ++l) {
                int32_t c = 0;
                for (int32_t s = 0; s < n; ++s)
                    c += (lvl[s] >= l);
                rec->active_count[l] = c;
            }
        rec->d_range[0] = range[0];
        rec->d_range[1] = range[1];
        for (int a = 0; a < 3; ++a)
            rec->dims[a] = dims[a];
    }

    for (size_t k = 0; k < 3 * (size_t)n; ++k) {
        xs[k] = (double)xs32[k];
        x0d[k] = (double)x0s[k];
    }
    /* The pre-stabilisation loop of Fig. 7: pre-stabilisation of the particles of level < S. */
    for (int32_t s = 0; s < n; ++s) {
        if (!(lvl[s] < p->stabil_s))
            continue;
        for (int32_t it = 0; it < p->stabil_iters; ++it) {
            double q[3] = {x0d[3 * s], x0d[3 * s + 1], x0d[3 * s + 2]};
            contact_obstacles(p, q);
            clamp_box(p, q);
            for (int a = 0; a < 3; ++a) {
                double d = q[a] - x0d[3 * s + a];
                x0d[3 * s + a] = q[a];
                xs[3 * s + a] += d;
            }
        }
    }
    /* The solver loop of Fig. 7: N_max Jacobi iterations over the active sets P_l. */
    for (int32_t l = 1; l <= p->n_max; ++l) {
#pragma omp parallel for schedule(static)
        for (int32_t s = 0; s < n; ++s) {
            int active = lvl[s] >= l;
            if (active || p->lambda_mode == ORC_LAMBDA_RECOMPUTE) {
                double rho;
                orc_constraint(p, n, xs, noff, nidx, s, &rho, NULL, NULL, &lam[s]);
                if (rec && rec->rho && l <= rec->rec_iters)
                    rec->rho[(size_t)(l - 1) * n + s] = active ? rho : NAN;
            } else {
                if (p->lambda_mode == ORC_LAMBDA_ZERO)
                    lam[s] = 0.0;
                if (rec && rec->rho && l <= rec->rec_iters)
                    rec->rho[(size_t)(l - 1) * n + s] = NAN;
            }
        }
        if (rec && rec->lam && l <= rec->rec_iters)
            memcpy(rec->lam + (size_t)(l - 1) * n, lam, sizeof(double) * (size_t)n);
#pragma omp parallel for schedule(static)
        for (int32_t s = 0; s < n; ++s)
            if (lvl[s] >= l)
                delta_p_one(p, xs, lam, noff, nidx, s, dp + 3 * s);
#pragma omp parallel for schedule(static)
        for (int32_t s = 0; s < n; ++s)
            if (lvl[s] >= l) {
                xs[3 * s + 0] += dp[3 * s + 0];
                xs[3 * s + 1] += dp[3 * s + 1];
                xs[3 * s + 2] += dp[3 * s + 2];
                contact_obstacles(p, xs + 3 * s);
                clamp_box(p, xs + 3 * s);
            }
        if (rec && rec->xs && l <= rec->rec_iters)
            memcpy(rec->xs + (size_t)(l - 1) * 3 * n, xs, sizeof(double) * 3 * (size_t)n);
    }

    /* The last step of Fig. 7: v = (x* - x) / dt, XSPH smoothing, x = x*. */
    for (int32_t s = 0; s < n; ++s)
        for (int a = 0; a < 3; ++a)
            vel[3 * s + a] = (xs[3 * s + a] - x0d[3 * s + a]) / (double)p->dt;
    orc_xsph(p, n, xs, vel, noff, nidx, vout);
    if (rec && rec->x_final)
        memcpy(rec->x_final, xs, sizeof(double) * 3 * (size_t)n);
    if (rec && rec->v_final)
        memcpy(rec->v_final, vout, sizeof(double) * 3 * (size_t)n);
    for (int32_t s = 0; s < n; ++s) {
        for (int a = 0; a < 3; ++a) {
            x[3 * s + a] = (float)xs[3 * s + a];
            v[3 * s + a] = (float)vout[3 * s + a];
        }
        id[s] = ids[s];
    }
    rc = 0;
done:
    free(level0);
    free(xpred);
    free(keys);
    free(order);
    free(start);
    free(xs32);
    free(x0s);
    free(ids);
    free(lvl);
    free(xs);
    free(dp);
    free(lam);
    free(vel);
    free(x0d);
    free(vout);
    free(noff);
    free(nidx);
    return rc;
}

/* Mean and maximum density deviation (the average-density plot of Fig. 9),
   with neighbours from the FP32 predicate at x and FP64 sums. */
int orc_density_stats(const orc_params *p, int32_t n, const float *x, double *rho_out, double stats[4])
{
    if (!p || n < 0 || (n > 0 && !x) || !stats || !(p->rho0 > 0.0f))
        return -1;
    stats[0] = stats[1] = stats[2] = stats[3] = 0.0;
    if (n == 0)
        return 0;
    int32_t *off = NULL, *idx = NULL;
    int rc = neighbors_alloc(p, n, x, &off, &idx);
    if (rc)
        return rc;
    double *xd = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!xd) {
        free(off);
        free(idx);
        return -3;
    }
    for (size_t k = 0; k < 3 * (size_t)n; ++k)
        xd[k] = (double)x[k];
    double *rho_all = rho_out ? rho_out : (double *)malloc(sizeof(double) * (size_t)n);
    if (!rho_all) {
        free(xd);
        free(off);
        free(idx);
        return -3;
    }
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i)
        orc_constraint(p, n, xd, off, idx, i, &rho_all[i], NULL, NULL, NULL);
    double s_abs = 0.0, s_max = 0.0, s_sgn = 0.0, s_pos = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        double e = rho_all[i] / (double)p->rho0 - 1.0;
        s_abs += fabs(e);
        if (fabs(e) > s_max)
            s_max = fabs(e);
        s_sgn += e;
        s_pos += e > 0.0 ? e : 0.0;
    }
    stats[0] = s_abs / n;
    stats[1] = s_max;
    stats[2] = s_sgn / n;
    stats[3] = s_pos / n;
    if (rho_all != rho_out)
        free(rho_all);
    free(xd);
    free(off);
    free(idx);
    return 0;
}
