/*
 * apbf.h -- C ABI of the GB300 (sm_103a) Adaptive Position-Based Fluids step.
 *
 * Method: Koster & Kruger, "Adaptive Position-Based Fluids: Improving
 * Performance of Fluid Simulations for Real-Time Applications", IJCGA 6(3),
 * 2016. One call of apbf_step() advances a scene by the simulation loop of
 * Fig. 7 (Sec. 5): external forces and prediction, neighbour discovery by a
 * counting-sort uniform grid with particle reordering (Sec. 6), N_max Jacobi
 * solver iterations of the density constraint (Eq. 4-7) in which particle i
 * is active only in iterations 1..N_i (Eq. 9-11), and the velocity/position
 * update. N_i is the particle's level of detail (Eq. 8) from its distance to
 * the camera (Sec. 4.1, DTC model) or from its distance behind the visible
 * surface of the particles rendered as spheres (Sec. 4.1 and Sec. 6, DTVS
 * model).
 *
 * Conventions for every entry point:
 *  - Returns apbf_status; nothing aborts, throws or exits.
 *  - "host" pointers are ordinary CPU memory owned by the caller and only
 *    read/written during the call (except apbf_read_positions_async, which
 *    fills its buffer after returning, by the next apbf_sync). "device"
 *    pointers are CUDA global memory.
 *  - Calls on one scene are not thread-safe; different scenes are independent.
 *  - All GPU work of a scene is issued on the stream given at creation, in
 *    call order (apbf_read_positions_async copies on a second stream of the
 *    library's, ordered after the step it reads and before any later reuse of
 *    its staging buffer). apbf_step() returns before the GPU finishes; a GPU-side error
 *    (e.g. a neighbour-list overflow) is reported by the next synchronising
 *    call (apbf_read_state, apbf_density_stats, apbf_sync, apbf_debug_read)
 *    and then sticks to the scene: every later call returns it.
 *  - Positions and velocities are FP32, 3 values per particle (x, y, z),
 *    in particle-id order (the order of apbf_scene_desc.pos). Inside a step
 *    the solver holds positions in fixed point: integers of u = 2^e metres
 *    relative to the grid origin, u the smallest power of two with 2^22 u >= h
 *    (so u <= h / 2^21) unless the grid spans 8e8 units or more on an axis
 *    (about 190 h), when u doubles until it does not. The neighbour search,
 *    the cell hash and the LOD use the FP32 positions themselves.
 */
#ifndef APBF_H
#define APBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define APBF_API __attribute__((visibility("default")))
#else
#define APBF_API
#endif

typedef enum apbf_status {
    APBF_OK = 0,
    APBF_ERR_INVALID_ARG = 1,       /* bad pointer, size, value or range (nothing was changed) */
    APBF_ERR_OUT_OF_MEMORY = 2,     /* device allocation failed, or the caller's arena is too small */
    APBF_ERR_CUDA = 3,              /* a CUDA runtime call failed (message in apbf_last_error) */
    APBF_ERR_TIMEOUT = 4,           /* a bounded device-side wait gave up */
    APBF_ERR_BAD_STATE = 5,         /* call not valid in the scene's current state */
    APBF_ERR_NEIGHBOR_OVERFLOW = 6, /* a particle had more neighbours than max_neighbors */
    APBF_ERR_NOT_SUPPORTED = 7,     /* option outside what the library implements */
    APBF_ERR_CHECK_FAILED = 8       /* an invariant check of the debug build failed (message: which, where) */
} apbf_status;

/* Level-of-detail models (Sec. 4.1). */
#define APBF_LOD_FIXED 0u /* plain PBF: every particle runs n_max iterations */
#define APBF_LOD_DTC 1u   /* distance to camera (Sec. 4.1) */
#define APBF_LOD_DTVS 2u  /* distance to the visible surface (Sec. 4.1, Sec. 6); single scenes, see apbf_set_view */

/* apbf_scene_desc.flags */
#define APBF_FLAG_NO_GRAPH 1u /* issue the step's kernels one by one instead of replaying a CUDA graph */

/*
 * Scene description. Units are SI (m, s, kg). Values are FP32 as the
 * solver uses them.
 *
 *  n            particles, 0 <= n < 2^31 - 1.
 *  pos, vel     host, 3n floats each in particle-id order; vel may be NULL (zero).
 *               Copied at creation; the caller keeps ownership.
 *  grid_lo/hi   static uniform-grid extent (cells of size h). Every particle
 *               must lie inside it. Cells per axis: floor((hi-lo)*(1/h)) + 1
 *               (FP32), at most 2047 (x, y) and 1023 (z).
 *  box_lo/hi    collision box (contacts, the collision response of Fig. 7), inside the grid extent.
 *  h            smoothing length = neighbour radius = cell size, > 0.
 *  dt           time step, > 0.
 *  mass         particle mass (uniform), > 0; w = 1/mass (Sec. 3).
 *  rho0         rest density (Eq. 5), > 0 (see apbf_rest_density).
 *  eps          relaxation added to the denominator of Eq. 4, >= 0.
 *  scorr_k, scorr_dq, scorr_n
 *               tensile term s_corr = -k (W(r)/W(dq))^n added to lambda_i +
 *               lambda_j in Eq. 7; k in m^2 (lambda's unit), 0 <= dq < h, n <= 16.
 *  xsph_c       XSPH viscosity, v_i += c sum_j (m/rho0) (v_j - v_i) W_ij.
 *  gravity      external acceleration f_ext (the external force of Fig. 7).
 *  n_min, n_max iteration range, 1 <= n_min <= n_max <= 255 (Eq. 8: levels 1..N_l).
 *  lod_mode     APBF_LOD_FIXED, APBF_LOD_DTC or APBF_LOD_DTVS (not in batches or servers:
 *               APBF_ERR_NOT_SUPPORTED).
 *  stabil_iters, stabil_s
 *               pre-stabilisation (Sec. 4.3, the pre-stabilisation loop of Fig. 7) of the set of
 *               Eq. 11 for l = S, i.e. the particles of level < S: before the
 *               solver, stabil_iters times (<= 64), each such particle's
 *               position at the start of the step is moved out of the
 *               obstacles (apbf_set_obstacles) and into the box, and its
 *               predicted position by the same amount, so its velocity gains
 *               nothing from the correction. S <= 1 (empty set) turns it off;
 *               S <= n_max.
 *  max_neighbors neighbour-list capacity per particle, 0 = 128, at most 255.
 *  flags        APBF_FLAG_*.
 */
typedef struct apbf_scene_desc {
    uint32_t n;
    const float *pos;
    const float *vel;
    float grid_lo[3], grid_hi[3];
    float box_lo[3], box_hi[3];
    float h, dt, mass, rho0, eps;
    float scorr_k, scorr_dq;
    uint32_t scorr_n;
    float xsph_c;
    float gravity[3];
    uint32_t n_min, n_max, lod_mode;
    uint32_t stabil_iters, stabil_s;
    uint32_t max_neighbors;
    uint32_t flags;
} apbf_scene_desc;

typedef struct apbf_scene apbf_scene;

/* Per-step counters of the last completed apbf_step (apbf_step_info). */
typedef struct apbf_step_info {
    uint64_t particle_iterations;   /* sum_i N_i = sum_l |P_l| (Eq. 10) */
    uint64_t neighbor_pairs;        /* sum_i |neighbours of i| */
    uint64_t lambda_pairs;          /* pairs visited by all lambda passes: sum_l sum_{i in P_l} |nbrs i| */
    uint32_t active_count[256];     /* |P_l| for l = 0..255 (l > n_max: 0) */
    float d_range[2];               /* distance range used by the LOD (0, 0 when fixed) */
    uint64_t total_particle_iterations; /* sum of particle_iterations over every apbf_step since the scene
                                           was created (kept on the device: reading it once at the end
                                           measures sum_i N_i over a run without a sync per step;
                                           apbf_autotune's trial steps do not count) */
} apbf_step_info;

/* Human-readable name of a status code (static string). */
APBF_API const char *apbf_status_string(apbf_status s);

/* Eq. 6 at an interior particle of a jitter-free cubic lattice of the given
 * spacing, self term included (poly6 kernel), computed on the host in FP64.
 * Host-only; needs no GPU. rho0 (host) receives the value. */
APBF_API apbf_status apbf_rest_density(float h, float mass, float spacing, double *rho0);

/* Device bytes a scene with this description needs (host-only, no GPU). */
APBF_API apbf_status apbf_scene_bytes(const apbf_scene_desc *desc, size_t *bytes);

/*
 * Create a scene on the current CUDA device.
 *  desc          host; validated (APBF_ERR_INVALID_ARG / NOT_SUPPORTED on failure).
 *  cuda_stream   a cudaStream_t of the current device (NULL = the legacy default stream).
 *  device_arena  device memory of at least apbf_scene_bytes() bytes, 256-byte
 *                aligned, owned by the caller and kept alive until
 *                apbf_destroy_scene; or NULL, in which case the library
 *                allocates (cudaMalloc) and frees it. A misaligned arena is
 *                APBF_ERR_INVALID_ARG, a short one APBF_ERR_OUT_OF_MEMORY;
 *                neither touches the GPU.
 *  arena_bytes   size of device_arena (ignored when NULL).
 *  out           host; receives the scene handle (NULL on failure).
 * Synchronises the stream once (the initial upload).
 */
APBF_API apbf_status apbf_create_scene(const apbf_scene_desc *desc, void *cuda_stream, void *device_arena,
                                       size_t arena_bytes, apbf_scene **out);

/*
 * Batches: several independent scenes stepped together, each stage of the
 * step one launch over all of them (their particles and grids concatenated).
 * A scene inside a batch evolves bit-identically to the same scene created
 * alone. Every scene's description must agree with scene 0 in everything but
 * n, pos, vel, grid_lo/hi and box_lo/hi (APBF_ERR_INVALID_ARG otherwise);
 * count <= 65535 and the total particle count < 2^31 - 1. A batch shares one
 * fixed-point unit: a scene whose grid needs a coarser unit than its h gives
 * (one spanning 8e8 units on an axis) steps alone (APBF_ERR_NOT_SUPPORTED).
 *  descs  host, count descriptions (copied, as for apbf_create_scene).
 * On a batch, apbf_set_camera / apbf_set_box set every scene (the _at forms
 * set one); apbf_read_state returns all particles, scene after scene, each
 * scene's particles in its own id order; apbf_density_stats and
 * apbf_get_step_info aggregate over all scenes (d_range: scene 0's).
 * apbf_create_scene(d, ...) is apbf_create_batch(d, 1, ...).
 */
APBF_API apbf_status apbf_batch_bytes(const apbf_scene_desc *descs, uint32_t count, size_t *bytes);
APBF_API apbf_status apbf_create_batch(const apbf_scene_desc *descs, uint32_t count, void *cuda_stream,
                                       void *device_arena, size_t arena_bytes, apbf_scene **out);
APBF_API apbf_status apbf_set_camera_at(apbf_scene *scene, uint32_t index, const float eye[3], const float dir[3],
                                        float d_near, float d_far);
APBF_API apbf_status apbf_set_box_at(apbf_scene *scene, uint32_t index, const float lo[3], const float hi[3]);

/* Camera of the DTC model (Sec. 4.1), used from the next apbf_step on.
 *  eye, dir  host, 3 floats; dir is stored for view-dependent models and must be finite.
 *  d_near < d_far: user-defined distance range; otherwise the range is the
 *  min/max camera distance over the scene at the start of each step (Sec. 4.1). */
APBF_API apbf_status apbf_set_camera(apbf_scene *scene, const float eye[3], const float dir[3], float d_near,
                                     float d_far);

/*
 * Camera image of the DTVS model (Sec. 4.1, Sec. 6), used from the next step
 * on; a DTVS scene must have one before it steps (APBF_ERR_BAD_STATE
 * otherwise); other scenes reject it (APBF_ERR_INVALID_ARG). The camera is a
 * pinhole at apbf_set_camera's eye looking along its dir: forward f =
 * dir/|dir|, right r = (f x up)/|f x up|, image up u = r x f; the image has
 * width x height pixels, row 0 at the top, and spans tan_half_fov (the
 * tangent of half the vertical field of view) vertically and tan_half_fov *
 * width/height horizontally at unit distance. Each step:
 *  1. every particle is rendered as a sphere of `radius` around its position:
 *     per pixel, the smallest positive distance along the ray through the
 *     pixel centre at which the ray enters a sphere (spheres containing the
 *     eye are not rendered);
 *  2. a particle whose centre projects into the image gets d = max(0,
 *     (|x - eye| - radius) - depth at that pixel), its distance behind the
 *     visible surface along its camera ray; visible particles get 0;
 *  3. N_i follows from d as for DTC (linear interpolation between the
 *     distance range, automatic over the particles in view, or the camera's
 *     d_near..d_far, and n_max..n_min); particles outside the view get n_min
 *     (or the level set by apbf_set_view_outside_level).
 * All of steps 1-3 is FP32 with every operation rounded (no contraction).
 *  width, height  1..16384 each, width * height <= 2^26.
 *  up             host, 3 floats, finite, not parallel to the camera's dir.
 * The image and its rasterisation lists (20 bytes per pixel, 20 per 8 x 8
 * tile, 81 per particle) are device memory the scene allocates here. */
APBF_API apbf_status apbf_set_view(apbf_scene *scene, uint32_t width, uint32_t height, float tan_half_fov,
                                   const float up[3], float radius);

/*
 * N_i of the DTVS particles outside the camera image, from the next step on.
 * The paper renders only what its camera sees and does not say which level an
 * unseen particle takes (Sec. 4.1); n_min (the default) gives unseen fluid the
 * least work, while a higher level keeps the density of fluid the camera sees
 * only in part closer to PBF with n_max iterations (Sec. 4.2: low levels left
 * without high-level neighbours drift in density). level: 0 (n_min) or
 * n_min..n_max; APBF_ERR_INVALID_ARG otherwise or for a scene that is not DTVS.
 */
APBF_API apbf_status apbf_set_view_outside_level(apbf_scene *scene, uint32_t level);

/*
 * Rigid obstacles (the paper's signed-distance-field obstacles of Sec. 6, here
 * analytic solids), used from the next step on by the collision response of
 * Fig. 7 -- after every position update of the solver, a predicted
 * position strictly inside an obstacle moves to the nearest point of its
 * surface (obstacles in order), then into the box -- and by the
 * pre-stabilisation above. The prediction itself is only clamped to the box.
 *  index      scene of a batch (0 for a single scene).
 *  obstacles  host, count entries (copied), count <= APBF_MAX_OBSTACLES; 0 removes them.
 *  kind       APBF_OBSTACLE_SPHERE: a = centre, b[0] = radius > 0.
 *             APBF_OBSTACLE_BOX: a solid block, a = min corner < b = max corner.
 *             APBF_OBSTACLE_CONE: a capped cone, a = centre of the base disc,
 *             axis +z, b[0] = base radius > 0, b[1] = height > 0.
 */
#define APBF_MAX_OBSTACLES 8u
#define APBF_OBSTACLE_SPHERE 1u
#define APBF_OBSTACLE_BOX 2u
#define APBF_OBSTACLE_CONE 3u

typedef struct apbf_obstacle {
    uint32_t kind;
    float a[3];
    float b[3];
} apbf_obstacle;

APBF_API apbf_status apbf_set_obstacles(apbf_scene *scene, uint32_t index, const apbf_obstacle *obstacles,
                                        uint32_t count);

/* Move the collision box (e.g. an oscillating wall) from the next step on.
 * lo, hi: host, 3 floats, grid_lo <= lo < hi <= grid_hi. */
APBF_API apbf_status apbf_set_box(apbf_scene *scene, const float lo[3], const float hi[3]);

/* Enqueue nsteps simulation steps (Fig. 7) on the scene's stream. Asynchronous. */
APBF_API apbf_status apbf_step(apbf_scene *scene, uint32_t nsteps);

/* Synchronise and copy the state to host buffers in particle-id order.
 * Each pointer may be NULL to skip it: pos, vel (3n floats), n_iter (n bytes:
 * the N_i of the last step, 0 before the first), rho (n floats: the density
 * of each particle's last lambda pass in the last step, 0 before the first). */
APBF_API apbf_status apbf_read_state(apbf_scene *scene, float *pos, float *vel, uint8_t *n_iter, float *rho);

/* Queue a copy of the positions (3n floats, particle-id order) to host memory
 * without waiting: the copy runs on a stream of its own, so it overlaps the
 * next apbf_step. pos should be pinned (page-locked) host memory; it is
 * complete once apbf_sync returns, and must stay valid until then. A later
 * readback waits for this copy before reusing the library's staging buffer.
 * Device errors are reported by the next synchronising call. */
APBF_API apbf_status apbf_read_positions_async(apbf_scene *scene, float *pos);

/* Synchronise and report density-error statistics of the current positions
 * (Fig. 9): stats (host, 4 doubles) = {mean |rho/rho0-1|, max |rho/rho0-1|,
 * mean (rho/rho0-1), mean max(0, rho/rho0-1)}, with a fresh neighbour search.
 * Does not change the simulation state. */
APBF_API apbf_status apbf_density_stats(apbf_scene *scene, double stats[4]);

/* Synchronise and return the counters of the last step (host struct). */
APBF_API apbf_status apbf_get_step_info(apbf_scene *scene, apbf_step_info *info);

/* Wait for the scene's queued work, asynchronous readbacks included; returns
 * the first error seen. */
APBF_API apbf_status apbf_sync(apbf_scene *scene);

/* Last error message of the scene (library-owned, valid until the next call
 * on the scene), or of the last failed create when scene is NULL. */
APBF_API const char *apbf_last_error(const apbf_scene *scene);

/* Release the scene and the memory it allocated (NULL-safe). Synchronises. */
APBF_API void apbf_destroy_scene(apbf_scene *scene);

/* ------------------------------------------- allocation-free diagnostic */

/* Limits of apbf_density_stats_static's built-in scratch memory. */
#define APBF_STATIC_MAX_PARTICLES 65536u
#define APBF_STATIC_MAX_CELLS 262144u

/*
 * The density-error statistics of apbf_density_stats, computed for positions
 * the caller already holds in device memory, without allocating any device
 * memory. (The paper has no counterpart: this is a convenience of the
 * library.) It is meant for callers that must not allocate GPU memory while
 * they run -- a game or renderer frame loop where cudaMalloc/cudaFree would
 * synchronise the device and stall the frame, a plug-in confined to its host
 * application's memory budget, or code with no allocator to hand to the
 * library.
 *
 *  pos        device, 3n floats (x, y, z per particle, any particle order).
 *  n          particles, at most APBF_STATIC_MAX_PARTICLES.
 *  h, mass, rho0, grid_lo, grid_hi (host, 3 floats each)
 *             as in apbf_scene_desc; the grid of cells of size h must have at
 *             most APBF_STATIC_MAX_CELLS cells. Positions outside the grid are
 *             counted in its boundary cells.
 *  stats      device, 4 doubles: {mean |rho/rho0-1|, max |rho/rho0-1|,
 *             mean (rho/rho0-1), mean max(0, rho/rho0-1)}, written
 *             asynchronously on cuda_stream (NULL = the legacy default stream).
 *  cuda_stream must belong to the current device (else APBF_ERR_INVALID_ARG;
 *             not checked while the stream is being captured into a CUDA graph,
 *             where the query would end the capture).
 * Larger n or grids return APBF_ERR_INVALID_ARG with a message in
 * apbf_last_error(NULL). The call makes no cudaMalloc, cudaFree or other
 * allocating call: all scratch (about 3.9 MB) is one static device array that
 * every GPU loading this library keeps until the process exits. The first call
 * on each device does the set-up: it looks up that array's device address and,
 * since CUDA loads a library's kernels lazily by default, that first lookup and
 * launch load the module, which reserves the array on the device then (an
 * implicit allocation that may synchronise). Make that first call once at
 * initialisation, outside any frame loop and before capturing any stream (a
 * first call on a capturing stream returns APBF_ERR_BAD_STATE); later calls
 * allocate nothing and may be captured into a CUDA graph. All calls share the one array and it keeps the
 * previous call's contents (the call clears what must start at zero), so calls
 * that overlap on the GPU -- on different streams, or from several host
 * threads -- race and must be serialised by the caller.
 */
APBF_API apbf_status apbf_density_stats_static(const float *pos, uint32_t n, float h, float mass, float rho0,
                                               const float grid_lo[3], const float grid_hi[3], double *stats,
                                               void *cuda_stream);

/* ---------------------------------------------------------------- timing */

/* Stage identifiers (timing and debug). */
#define APBF_STAGE_LOD_RANGE 0u  /* a1: DTVS depth image, distances and their range (empty for the
                                    other LOD models) */
#define APBF_STAGE_PREDICT 1u    /* a1-a4: camera-distance range, prediction, cell hash, histogram */
#define APBF_STAGE_SCAN 2u       /* a4/a6: exclusive scan = cell start/end */
#define APBF_STAGE_SCATTER 3u    /* a4: slot scatter */
#define APBF_STAGE_REORDER 4u    /* a1, a4/a5: level, stable rank and reorder */
#define APBF_STAGE_NEIGHBORS 5u  /* neighbour lists (the neighbour search of Fig. 7); with levels, it
                                    also places each particle in the active list (a7) */
#define APBF_STAGE_LEVELS 6u     /* a7: active-set sizes and offsets per level and tile (runs before
                                    the neighbour search) */
#define APBF_STAGE_LAMBDA 7u     /* a8 */
#define APBF_STAGE_DELTAP 8u     /* a9 */
#define APBF_STAGE_FINALIZE 9u   /* a10 */
#define APBF_STAGE_PRESTAB 10u   /* pre-stabilisation (the pre-stabilisation loop of Fig. 7), between LEVELS and LAMBDA */
#define APBF_STAGE_COUNT 11u

/* Enable (1) or disable (0) per-stage CUDA-event timing of apbf_step. While
 * enabled, steps are issued kernel by kernel (no graph replay). */
APBF_API apbf_status apbf_set_timing(apbf_scene *scene, int enable);

/* Synchronise and report, per stage (APBF_STAGE_COUNT entries each, host):
 * the summed device time in ms and the number of kernel launches timed since
 * the last report; then reset the counters. */
APBF_API apbf_status apbf_timing_report(apbf_scene *scene, double *ms, uint64_t *launches);

/* ------------------------------------------------------------- tuning */

/* Result of apbf_autotune: the chosen configuration and every trial. */
typedef struct apbf_tune_result {
    uint32_t block;          /* threads per block of the solver passes (128 or 256) */
    float mask_threshold;    /* masked (all particles) instead of compacted when |P_l| >= threshold * n */
    double ms_per_step;      /* the chosen configuration's trial time */
    uint32_t tried;          /* trials below */
    uint32_t blocks[16];
    float thresholds[16];
    double ms[16];
} apbf_tune_result;

/* Set the solver passes' launch configuration: block = 128 or 256 threads;
 * iterations with a shrinking active set run over all particles (masked)
 * instead of the compacted list when |P_l| >= mask_threshold * n (a
 * threshold above 1 means always compacted). Results do not depend on it. */
APBF_API apbf_status apbf_set_tuning(apbf_scene *scene, uint32_t block, float mask_threshold);

/* Time every configuration (2 blocks x 5 thresholds) over trial_steps steps
 * each (1..1000, after 2 warm-up steps) from the current state, restore the
 * state, and keep the fastest. out (host) receives the choice and the trials.
 * Synchronises; the state and the results of later steps are unchanged. */
APBF_API apbf_status apbf_autotune(apbf_scene *scene, uint32_t trial_steps, apbf_tune_result *out);

/* ------------------------------------------------------------- serving */

/*
 * A server steps many independent scenes that arrive and leave over time (the
 * paper's real-time setting, Sec. 1 and Sec. 7, with one simulation per client
 * instead of one per application). Requests wait in a FIFO queue and are
 * admitted, in arrival order, into one resident device pool while the pool's
 * particle, cell and scene capacities have room; a request that does not fit
 * waits (no later request overtakes it). Each apbf_server_tick() advances every
 * resident scene by one step of Fig. 7, all of them in one batched step (one
 * launch per stage). A scene leaves the pool at the first tick after its last
 * step, when its final state is copied to the caller's buffers. A scene's
 * result is bit-identical to the same scene stepped alone with
 * apbf_create_scene / apbf_set_camera(eye, auto range) / apbf_step(steps).
 * Every request must agree with the server's physics description in
 * everything but n, pos, vel, grid_lo/hi and box_lo/hi. Calls on one server
 * are not thread-safe. A device error of the pool (neighbour-list overflow,
 * CUDA error) fails every resident request and sticks to the server.
 */
typedef struct apbf_server apbf_server;

typedef struct apbf_server_desc {
    const apbf_scene_desc *physics; /* host: h, dt, mass, rho0, eps, s_corr, XSPH, gravity, n_min/n_max,
                                       lod_mode, max_neighbors, flags shared by every request (its n, pos,
                                       vel, grid and box are ignored) */
    uint32_t max_particles;         /* resident particle capacity (< 2^31 - 1); 0 = the most that budget_bytes holds */
    uint32_t max_cells;             /* resident grid-cell capacity (< 2^31); 0 = 4 x max_particles */
    uint32_t max_scenes;            /* resident scenes (<= 65535); 0 = 4096 */
    size_t budget_bytes;            /* device bytes the pool may use; 0 = no limit (max_particles required) */
    double target_step_ms;          /* step-latency target of admission; 0 = off (admit while the pool has
                                       room). When > 0, a queued request is admitted only while the resident
                                       particles times the measured cost per particle-step stay below 0.9 x
                                       this target (a request is always admitted into an empty pool). The
                                       cost is a running average of the device time per particle of the
                                       ticks that stepped at least 262144 particles, 2 ns before the first. */
} apbf_server_desc;

typedef struct apbf_request {
    const apbf_scene_desc *scene;   /* host; n >= 1, pos, vel (may be NULL), grid, box copied at submit */
    float eye[3];                   /* DTC camera position (automatic distance range, Sec. 4.1) */
    uint32_t steps;                 /* steps to run, >= 1 */
    float *pos_out, *vel_out;       /* host, 3n floats each in particle-id order, or NULL; written by the tick
                                       that retires the request; the caller keeps them valid until then */
    const apbf_obstacle *obstacles; /* host, n_obstacles entries (copied at submit; as apbf_set_obstacles), or NULL */
    uint32_t n_obstacles;           /* <= APBF_MAX_OBSTACLES */
} apbf_request;

typedef struct apbf_tick_info {
    uint64_t tick;                  /* index of this tick (0, 1, ...) */
    uint32_t resident_scenes;       /* scenes stepped by this tick */
    uint32_t resident_particles;    /* their particles */
    uint32_t admitted;              /* requests admitted by this tick */
    uint32_t completed;             /* requests retired (results written) by this tick */
    uint32_t queued;                /* requests still waiting */
    uint32_t failed;                /* requests retired as failed by this tick (see apbf_request_info.status) */
    double prev_step_ms;            /* device time of the previous tick's step (0 if it stepped nothing) */
    uint64_t total_particle_iterations; /* sum_i N_i over every step the pool completed so far */
    uint32_t particle_limit;        /* resident particles admission allows now (capacity, or the latency target's) */
    uint32_t pad;
} apbf_tick_info;

#define APBF_REQ_QUEUED 0u
#define APBF_REQ_RESIDENT 1u
#define APBF_REQ_DONE 2u
#define APBF_REQ_FAILED 3u

typedef struct apbf_request_info {
    uint32_t state;                 /* APBF_REQ_* */
    uint32_t steps_done;
    uint32_t n, steps;
    uint64_t submit_tick, admit_tick, done_tick; /* tick counter at submit, admission, retirement */
    apbf_status status;             /* APBF_REQ_FAILED: why; APBF_ERR_NEIGHBOR_OVERFLOW when one of its
                                       particles had more neighbours than max_neighbors (only that request
                                       fails: the other resident scenes' lists are their own) */
    uint32_t pad;
} apbf_request_info;

/* Pool bytes and resolved capacities of a description (host-only, no GPU);
 * each output may be NULL. APBF_ERR_OUT_OF_MEMORY if the capacities exceed
 * budget_bytes. */
APBF_API apbf_status apbf_server_bytes(const apbf_server_desc *desc, size_t *bytes, uint32_t *max_particles,
                                       uint32_t *max_cells);

/* Create a server on the current device; its pool is allocated (cudaMalloc)
 * once, here. cuda_stream as in apbf_create_scene. */
APBF_API apbf_status apbf_server_create(const apbf_server_desc *desc, void *cuda_stream, apbf_server **out);

/* Queue a request (validated and copied; APBF_ERR_INVALID_ARG if it could never
 * fit the pool alone; APBF_ERR_NOT_SUPPORTED if its grid needs a coarser
 * fixed-point unit than the pool's, as for batches). ticket (host) receives
 * its id. Does not touch the GPU. */
APBF_API apbf_status apbf_server_submit(apbf_server *server, const apbf_request *req, uint64_t *ticket);

/* One tick: wait for the previous tick's step, retire the scenes it finished
 * (results to their buffers) and the scenes whose particles overflowed their
 * neighbour lists in it (APBF_REQ_FAILED, no results; the other scenes go on
 * unaffected), close the pool's gaps, admit queued requests in arrival order
 * (while the pool has room and, with target_step_ms, while the step stays
 * within the latency target), and enqueue one step of every resident scene
 * (returns before it finishes). info (host, may be NULL) receives the tick's
 * counts. */
APBF_API apbf_status apbf_server_tick(apbf_server *server, apbf_tick_info *info);

/* State of a request (host output). */
APBF_API apbf_status apbf_server_query(apbf_server *server, uint64_t ticket, apbf_request_info *info);

/* Last error message of the server (or of the last failed create when NULL). */
APBF_API const char *apbf_server_last_error(const apbf_server *server);

/* Release the server (NULL-safe); synchronises. Unfinished requests are dropped. */
APBF_API void apbf_server_destroy(apbf_server *server);

/* ----------------------------------------------------- test-only exports */

/* Run one fresh step of the current state up to and including a stage
 * (iteration 1..n_max for LAMBDA / DELTAP). The state (positions, velocities,
 * order) is not advanced unless stage == APBF_STAGE_FINALIZE. */
APBF_API apbf_status apbf_debug_step_to(apbf_scene *scene, uint32_t stage, uint32_t iteration);

#define APBF_DBG_KEYS 0u          /* u32[n]  cell key, pre-sort (state) order */
#define APBF_DBG_STATE_IDS 1u     /* u32[n]  particle ids in state order */
#define APBF_DBG_LEVEL_PRESORT 2u /* u8[n]   N_i, pre-sort order (from APBF_STAGE_REORDER on) */
#define APBF_DBG_SORTED_IDS 3u    /* u32[n]  particle ids in sorted order */
#define APBF_DBG_CELL_START 4u    /* u32[ncell+1] */
#define APBF_DBG_XPRED 5u         /* float4[n] predicted positions (FP32), sorted */
#define APBF_DBG_LEVEL 6u         /* u8[n]   N_i, sorted */
#define APBF_DBG_NBR_COUNT 7u     /* u8[n]   neighbour count, sorted */
#define APBF_DBG_NBR 8u           /* u32[max_neighbors*n]: entry k of particle p at k*n+p, the
                                     neighbour's sorted slot; n pads a list to a multiple of 4 */
#define APBF_DBG_ACTIVE 9u        /* u32[n]  sorted slots, active-set order (P_l = prefix; from
                                     APBF_STAGE_NEIGHBORS on) */
#define APBF_DBG_LEVEL_COUNT 10u  /* u32[n_max+2] |P_l|, l = 0..n_max+1 */
#define APBF_DBG_LAMBDA 11u       /* float[n] lambda after the stage, sorted */
#define APBF_DBG_RHO 12u          /* float[n] density of the last lambda pass, sorted */
#define APBF_DBG_XSTAR 13u        /* float4[n] current x* (absolute FP32), sorted */
#define APBF_DBG_DRANGE 14u       /* float[2*scenes] LOD distance ranges: the minima, then the maxima */
#define APBF_DBG_DEPTH 15u        /* float[width*height] DTVS depth image (0x7f7f7f7f bits: empty) */
#define APBF_DBG_LOD_DISTANCE 16u /* float[n] DTVS distance behind the visible surface, pre-sort
                                     (state) order; -1 outside the view */

/* Copy a debug field (see APBF_DBG_*) to host memory of `bytes` bytes
 * (must equal the field's size). Synchronises. */
APBF_API apbf_status apbf_debug_read(apbf_scene *scene, uint32_t field, void *host, size_t bytes);

/* Sizes of the scene's grid: dims (3 ints), ncell, max_neighbors (host outputs). */
APBF_API apbf_status apbf_debug_dims(apbf_scene *scene, int32_t dims[3], uint32_t *ncell,
                                     uint32_t *max_neighbors);

/*
 * Debug build (libapbf_debug.so, compiled with APBF_DEBUG_CHECKS=1; the
 * paper has no counterpart): every step also checks, on the device, that each
 * cell key lies in its grid, that the cell counts add up to the particle count,
 * that each particle's sorted slot lies in its cell's range, that |P_l| <= n and
 * |P_l| <= |P_(l-1)|, and that every neighbour entry names a particle (or the
 * padding record). A failure keeps the guarded access inside its array, and
 * the next synchronising call returns APBF_ERR_CHECK_FAILED (sticky) naming the
 * first failed check and its index. The release build has none of these.
 */
/* 1 in the debug build, 0 in the release build. */
APBF_API int apbf_debug_checks_enabled(void);

/* Debug build only (APBF_ERR_NOT_SUPPORTED otherwise): with what = 1, every
 * later step's neighbour search writes one entry that names the record past the
 * padding one (still inside the scene's memory), which the checks must catch;
 * what = 0 stops it. A test of the checks themselves. */
APBF_API apbf_status apbf_debug_plant(apbf_scene *scene, uint32_t what);

#ifdef __cplusplus
}
#endif
#endif /* APBF_H */
