/*
 * apbf_oracle.h -- plain, slow CPU reference of one Adaptive Position-Based
 * Fluids time step (Koster & Kruger 2016, Sec. 3-5, Fig. 7).
 *
 * TEST INFRASTRUCTURE ONLY. This library is called by the tests, by the
 * package's smoke check and by the benchmark's CPU-baseline leg. The product
 * path (the CUDA library) never links, loads or calls it, and the two share
 * no code.
 *
 * Precision: every integer decision of the step (LOD level, cell index,
 * neighbour predicate) and the prediction that feeds it are evaluated in
 * IEEE FP32 operation by operation (no contraction), because the scene's
 * state is FP32 and these decisions must be reproducible exactly. The solver
 * arithmetic (density, lambda, position corrections, velocity, XSPH) runs in
 * FP64 from the FP32 values; the new state is rounded to FP32 at the end of
 * the step.
 *
 * Return codes: 0 ok, -1 invalid argument, -2 caller capacity too small,
 * -3 allocation failure.
 */
#ifndef APBF_ORACLE_H
#define APBF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_LOD_FIXED 0
#define ORC_LOD_DTC 1
#define ORC_LOD_DTVS 2

#define ORC_LAMBDA_STALE 0     /* inactive neighbours keep their last lambda */
#define ORC_LAMBDA_ZERO 1      /* inactive neighbours contribute lambda = 0 */
#define ORC_LAMBDA_RECOMPUTE 2 /* lambda recomputed for every particle each iteration */

/* Camera image of the DTVS model (Sec. 4.1, Sec. 6): a pinhole camera at
   orc_params.eye looking along dir, world up `up`, vertical half-angle with
   tangent tan_half_fov, width x height pixels (row 0 at the top); particles
   are rendered as spheres of the given radius. */
typedef struct orc_view {
    int32_t width, height;
    float tan_half_fov;
    float dir[3];
    float up[3];
    float radius;
    int32_t brute_force; /* 1: test every pixel against every sphere (no bounding box) */
    int32_t outside_level; /* N_i of a particle outside the view; 0: n_min (reading 20) */
} orc_view;

/* Rigid obstacles (Sec. 6 uses signed-distance fields; these are analytic
   solids): a point strictly inside is moved to the nearest point of the
   solid's surface. */
#define ORC_MAX_OBSTACLES 8
#define ORC_OBSTACLE_SPHERE 1 /* a = centre, b[0] = radius */
#define ORC_OBSTACLE_BOX 2    /* a = min corner, b = max corner (a solid block) */
#define ORC_OBSTACLE_CONE 3   /* a = centre of the base disc, axis +z, b[0] = base radius, b[1] = height */

typedef struct orc_obstacle {
    int32_t kind;
    float a[3];
    float b[3];
} orc_obstacle;

typedef struct orc_params {
    /* Scene values exactly as the solver receives them (FP32). */
    float h, dt, mass, rho0, eps, scorr_k, scorr_dq, xsph_c;
    int32_t scorr_n;
    float gravity[3];
    float grid_lo[3], grid_hi[3]; /* static uniform-grid extent */
    float box_lo[3], box_hi[3];   /* collision box of this step (inside the grid) */
    int32_t n_min, n_max, lod_mode;
    float eye[3];
    float d_near, d_far;          /* d_near >= d_far: automatic range */
    int32_t lambda_mode;          /* ORC_LAMBDA_* */
    int32_t lod_rounding;         /* 0: equal-width bins, 1: rounded interpolation */
    orc_view view;                /* DTVS only */
    /* Pre-stabilisation (Sec. 4.3, the pre-stabilisation loop of Fig. 7): particles of level < stabil_s
       (the set of Eq. 11 for l = S) are moved out of the obstacles and into the box
       stabil_iters times before the solver, current and predicted positions alike. */
    int32_t stabil_iters, stabil_s;
    int32_t n_obstacles;
    orc_obstacle obstacles[ORC_MAX_OBSTACLES];
} orc_params;

typedef struct orc_record {
    /* Optional outputs of one step (NULL = not recorded), caller-owned.
       "pre-sort order" is the state order at the start of the step;
       "sorted order" is the order after the counting sort (by cell key, ties
       by particle id), which is also the state order after the step. */
    float *xpred;           /* 3n, pre-sort order, FP32 prediction incl. box clamp */
    int32_t *level_presort; /* n, pre-sort order */
    uint32_t *keys;         /* n, pre-sort order */
    int32_t *order;         /* n, sorted slot -> pre-sort index */
    uint32_t *cell_start;   /* ncell + 1 */
    int64_t cell_cap;       /* capacity of cell_start */
    int32_t *nbr_off;       /* n + 1, CSR over sorted slots */
    int32_t *nbr_idx;       /* neighbour sorted slots */
    int64_t nbr_cap;        /* capacity of nbr_idx */
    int32_t *active_count;  /* n_max + 2 entries: |P_l|, l = 0 .. n_max + 1 */
    int32_t rec_iters;      /* record iterations 1 .. rec_iters of lam/rho/xs */
    double *lam;            /* rec_iters * n, sorted: lambda after the lambda pass of iteration l */
    double *rho;            /* rec_iters * n, sorted: density at iteration l (NaN if inactive) */
    double *xs;             /* rec_iters * 3n, sorted: x* after the update of iteration l */
    double *x_final;        /* 3n, sorted: new position before rounding */
    double *v_final;        /* 3n, sorted: new velocity before rounding */
    float d_range[2];       /* out: distance range used by the LOD */
    int32_t dims[3];        /* out: grid cells per axis */
} orc_record;

/* SPH kernels (Eq. 6 uses W; Eq. 7 uses grad W): poly6 and spiky. */
double orc_poly6(double r2, double h);
double orc_spiky(double r, double h);
void orc_spiky_grad(const double r[3], double h, double g[3]);

/* Density of an interior particle of a jitter-free cubic lattice. */
double orc_rest_density(double h, double mass, double spacing);

/* Grid cells per axis: floor((hi - lo) * inv_h) + 1 in FP32, inv_h = 1/h in FP32. */
int orc_grid_dims(const orc_params *p, int32_t dims[3]);

/* DTVS camera basis: forward f = dir/|dir|, right r = (f x up)/|f x up|,
   image up u = r x f (FP32). Returns -1 when dir or f x up is zero. */
int orc_view_basis(const orc_view *v, float f[3], float r[3], float u[3]);

/* Unit direction of the camera ray through the centre of pixel (px, py) (FP32). */
int orc_pixel_ray(const orc_view *v, int32_t px, int32_t py, float ray[3]);

/* Depth image of the particles rendered as spheres (Sec. 6): per pixel the
   smallest positive distance along the pixel's ray to the surface of a sphere
   it enters, or the value with bit pattern 0x7f7f7f7f (3.4e38) where it
   enters none. width*height floats. */
int orc_depth_image(const orc_params *p, int32_t n, const float *x, float *depth);

/* DTVS distance (Sec. 4.1): for a particle whose centre projects into the
   image, max(0, (|x - eye| - radius) - depth at that pixel), the distance
   behind the visible surface along its camera ray; -1 for particles outside
   the view. */
int orc_dtvs_distance(const orc_params *p, int32_t n, const float *x, const float *depth, float *dist);

/* Sec. 4.1 DTC / DTVS model + Eq. 8: per-particle level from the camera
   distance (DTC) or the distance behind the visible surface (DTVS;
   particles outside the view get n_min, or view.outside_level when that is
   set, and do not enter the automatic range). */
int orc_lod_levels(const orc_params *p, int32_t n, const float *x, int32_t *level, float range[2]);

/* Nearest surface point of an obstacle for a point strictly inside it (FP64);
   returns 1 and writes q when x is inside, 0 (q = x) otherwise. */
int orc_obstacle_project(const orc_obstacle *o, const double x[3], double q[3]);

/* The prediction step of Fig. 7 plus the box clamp, FP32. */
int orc_predict(const orc_params *p, int32_t n, const float *x, const float *v, float *xpred);

/* Cell index of each position (FP32). */
int orc_cell_keys(const orc_params *p, int32_t n, const float *xpos, uint32_t *keys);

/* Stable counting sort by key: order[slot] = input index; cell_start has ncell + 1 entries. */
int orc_counting_sort(int32_t n, const uint32_t *keys, int64_t ncell, int32_t *order, uint32_t *cell_start);

/* Neighbour sets {j != i : |x_i - x_j|^2 < h^2} (FP32 predicate) by a cell
   list, reported in input indices, each list ascending. */
int orc_neighbors(const orc_params *p, int32_t n, const float *x, int32_t *off, int32_t *idx, int64_t cap);

/* Eq. 4-6 for particle i: density, constraint value, gradients
   grad[0..2] = d C_i / d x_i and grad[3(k+1)..] = d C_i / d x_{nbr k}, and lambda. */
int orc_constraint(const orc_params *p, int32_t n, const double *xs, const int32_t *nbr_off,
                   const int32_t *nbr_idx, int32_t i, double *rho, double *C, double *grad,
                   double *lambda);

/* Eq. 7 with the tensile term for every particle (no clamp). */
int orc_delta_p(const orc_params *p, int32_t n, const double *xs, const double *lam,
                const int32_t *nbr_off, const int32_t *nbr_idx, double *dp);

/* XSPH velocity smoothing over the given neighbour sets. */
int orc_xsph(const orc_params *p, int32_t n, const double *xs, const double *v,
             const int32_t *nbr_off, const int32_t *nbr_idx, double *vout);

/* One APBF step (Fig. 7). x, v (3n) and id (n, a permutation of 0..n-1)
   are the state in its current order; on return they hold the new state in
   sorted order (cell key, then particle id). The result does not depend on
   the order of the input. */
int orc_step(const orc_params *p, int32_t n, float *x, float *v, int32_t *id, orc_record *rec);

/* Threads of the per-particle loops (OpenMP; <= 0 keeps the current count).
   Returns the count now in use (1 when built without OpenMP). Results are
   bit-identical at any thread count. */
int orc_set_threads(int32_t nthreads);

/* Density diagnostic at the given positions (fresh neighbour search):
   stats = {mean |rho/rho0-1|, max |rho/rho0-1|, mean (rho/rho0-1), mean max(0, rho/rho0-1)}. */
int orc_density_stats(const orc_params *p, int32_t n, const float *x, double *rho, double stats[4]);

#ifdef __cplusplus
}
#endif
#endif
