// Internal types of the CUDA implementation of include/apbf.h.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "apbf.h"

namespace apbf {

constexpr uint32_t kDefaultMaxNeighbors = 128;
// Particles of a scene, batch or pool: below 2^31, so that a neighbour entry (a
// plain 32-bit sorted slot) can also name the padding record n.
constexpr uint32_t kMaxParticles = 0x7fffffffu;
// Neighbour entries are stored in blocks of kEntryBlock per particle: entry k
// of list column t at ((k / 4) * n + t) * 4 + k % 4, so a thread reads a
// block with one 16-byte load and a warp's block loads are contiguous. Lists
// are padded to whole blocks with an entry naming slot n, a record placed far
// outside every grid (the record arrays hold n + 1 entries), so the solver
// reads whole blocks without bounds checks.
constexpr uint32_t kEntryBlock = 4;
constexpr uint32_t kListPad = kEntryBlock;
__host__ __device__ inline size_t entry_index(uint32_t k, size_t t, size_t n)
{
    return ((size_t)(k / kEntryBlock) * n + t) * kEntryBlock + k % kEntryBlock;
}
__host__ __device__ constexpr uint32_t list_rows(uint32_t max_nbr)
{
    return (max_nbr + kListPad - 1) / kListPad * kListPad;
}
constexpr int kBlock = 256;          // threads per block of the per-particle kernels
constexpr int kScanTile = 4096;      // cells per block of the grid scan (1024 threads x 4)
#ifndef APBF_PREDICT_BLOCKS
#define APBF_PREDICT_BLOCKS 1024
#endif
constexpr unsigned kPredictBlocks = APBF_PREDICT_BLOCKS;  // grid cap of a single scene's predict pass (its range atomics)
constexpr int kLevelTile = kBlock;   // sorted slots per tile of the active-set partition (a block of the neighbour search)

// Tiles of the active-set partition for n particles, rounded up to a multiple
// of 4 (the level scan reads the per-tile counts four at a time; the extra
// tiles hold no particle and count zero).
inline uint32_t level_tile_count(uint64_t n) { return (uint32_t)(((n + kLevelTile - 1) / kLevelTile + 3) / 4 * 4); }
constexpr int kTilePx = 8;           // DTVS depth tiles: kTilePx x kTilePx pixels, one block each
constexpr uint32_t kMaxSplatTiles = 4096;  // spheres covering more tiles take the big-sphere path
constexpr int kBigBlockPx = 64;            // image blocks of the big-sphere path
constexpr uint32_t kSplatChunk = 1024;     // list entries per work chunk of the tile rasteriser
constexpr uint32_t kSplatListPerParticle = 16;  // tile-list capacity: 16 entries per particle + 65536
constexpr uint8_t kFrontNeighbors = 28;    // phase-0 spheres: fewer neighbours than this in the last step

// Fixed-point solver positions: every scene's positions, in units of
// StepConst::fx_u relative to its grid origin, must span fewer than kFxSpan
// units, so that the difference of any two of them, biased by kFxMagic, is the
// bit pattern of a finite float (see kernels.cu).
constexpr double kFxSpan = 8.0e8;
constexpr int32_t kFxMagic = 0x4B400000;  // bit pattern of 1.5 * 2^23
constexpr int32_t kFxFar = -(1 << 30);    // the padding record: at least 3h from every particle

// Device error word bits.
constexpr uint32_t kErrNeighborOverflow = 1u;
constexpr uint32_t kErrDebugCheck = 2u;  // a debug-build invariant check failed (see APBF_DEBUG_CHECKS)

// Debug-build invariant checks (compiled in with -DAPBF_DEBUG_CHECKS=1; the
// release library has none). A failed check sets kErrDebugCheck, records the
// first failure's code and index in Buffers::dbg (dbg[0], dbg[1]) and keeps
// the access it guards inside its array. dbg[2] != 0 asks the neighbour
// search to plant one out-of-range entry (a test of the checks themselves).
#ifndef APBF_DEBUG_CHECKS
#define APBF_DEBUG_CHECKS 0
#endif
constexpr uint32_t kCheckCellKey = 1u;      // a cell key outside the scene's grid
constexpr uint32_t kCheckScanTotal = 2u;    // the cell counts do not add up to the particle count
constexpr uint32_t kCheckSortedSlot = 3u;   // a particle's sorted slot outside its cell's range
constexpr uint32_t kCheckActiveCount = 4u;  // |P_l| above n or above |P_(l-1)|
constexpr uint32_t kCheckNeighbor = 5u;     // a neighbour entry naming a slot beyond the padding record

// Slots of the 64-bit counters: [0] neighbour pairs of the step without a
// level partition, [2 + bin] pairs per level bin with one (reset each step), two slots of scratch for the density
// diagnostic, and the running total of particle-iterations (sum_l |P_l|, Eq.
// 10) over every completed step, which nothing resets (the autotuner keeps a
// copy in the slot after it while its trial steps run).
constexpr uint32_t kDiagCounterSlot = 2 + 256;
constexpr uint32_t kIterTotalSlot = kDiagCounterSlot + 2;
constexpr uint32_t kIterSaveSlot = kIterTotalSlot + 1;
constexpr uint32_t kCounterSlots = kIterSaveSlot + 1;

// Step constants, fixed for a scene's lifetime (passed by value as kernel
// arguments and therefore baked into the captured step graph).
struct StepConst {
    uint32_t n;
    uint32_t ncell;
    int32_t nx, ny, nz;
    float glo[3];
    float inv_h;        // fl(1/h), the cell-hash scale
    float h;
    float h2;           // fl(h*h): the FP32 neighbour predicate bound
    float dt, inv_dt;
    float g[3];
    // Solver positions in fixed point (see kernels.cu): integers of the unit
    // fx_u = 2^fx_e metres, relative to the scene's grid origin; 2^22 fx_u >= h.
    float fx_u, fx_inv_u;
    float fx_off;       // -1.5 * 2^23 * fx_u: with the bias kFxMagic, one FMA turns a difference into metres
    int32_t fx_e;
    // solver coefficients (FP32 from FP64 host values)
    float mass_poly6;   // m * 315 / (64 pi h^9)
    float h6;           // (h^2)^3: self term of the density sum
    float inv_rho0;
    float c_lam;        // w (m * 45/(pi h^6) / rho0)^2
    float eps;
    float c_dp;         // -(w m / rho0) * 45/(pi h^6)
    float c_dpu;        // c_dp / fx_u: the correction in fixed-point units
    float v_scale;      // fx_u / dt: velocity of a displacement of one unit
    float inv_wdq;      // 1 / (h^2 - dq^2)
    float neg_k;        // -k
    uint32_t scorr_n;
    float c_xsph;       // c (m / rho0) * 315/(64 pi h^9)
    uint32_t n_min, n_max, K, lod_mode;
    uint32_t dtvs_outside;  // DTVS: N_i of a particle outside the view (n_min unless set)
    uint32_t max_nbr;
    uint32_t level_tiles;
    float rho0;         // rest density as given (FP32)
    uint32_t stabil_s, stabil_iters;  // pre-stabilisation of the levels below S (Sec. 4.3), S <= 1: off
    uint32_t scenes;    // scenes in the batch (1: the fields glo, nx.., m above describe it)
};

// Geometry of one scene of a batch (device table, one entry per scene). The
// scenes' particles and cells are concatenated: scene s owns particle slots
// p0 .. p0+n-1 (in every order the step uses, because cell keys are
// scene-major) and cell keys cell_base .. cell_base + nx*ny*nz - 1.
struct SceneGeom {
    float glo[3];
    int32_t nx, ny, nz;
    uint32_t cell_base;
    uint32_t p0, n;
};

// Per-step values that callers change between steps (device copy read by kernels,
// one per scene).
// A rigid obstacle (apbf_obstacle): sphere (a = centre, b[0] = radius), solid
// block (a = min, b = max corner) or capped cone (a = base centre, axis +z,
// b[0] = base radius, b[1] = height).
struct Obstacle {
    uint32_t kind;
    float a[3];
    float b[3];
    uint32_t pad;
};

struct DynParams {
    float box_lo[4];
    float box_hi[4];
    float eye[4];
    float dir[4];  // viewing direction (DTVS)
    float d_near, d_far;
    uint32_t auto_range;
    uint32_t n_obst;  // obstacles in use
    Obstacle obst[APBF_MAX_OBSTACLES];
};

// Camera image of the DTVS model (Sec. 4.1, Sec. 6), fixed between
// apbf_set_view calls (passed by value, so it is part of the captured step).
struct ViewConst {
    uint32_t W = 0, H = 0;
    float tan_half = 0.0f;  // tan of half the vertical field of view
    float up[3] = {0.0f, 0.0f, 1.0f};
    float radius = 0.0f;    // sphere radius of the rendered particles
    // frustum cull: cos and sin of gamma + 0.01, gamma the angle between the
    // view direction and an image corner's ray (cos = -1e30 turns it off)
    float cull_cos = -1.0e30f, cull_sin = 0.0f;
    uint32_t *depth = nullptr;  // W*H float bits, row 0 at the top
    float4 *ray = nullptr;      // W*H unit pixel rays of the current camera
    // binning of the rendered spheres into kTilePx x kTilePx pixel tiles
    uint32_t tiles_x = 0, tiles_y = 0;
    uint32_t *tile_cnt = nullptr;    // spheres per tile
    uint32_t *tile_fill = nullptr;   // fill counters of the scatter pass
    uint32_t *tile_start = nullptr;  // tiles + 1 list offsets
    uint32_t *chunk_start = nullptr; // tiles + 1 offsets of the tiles' kSplatChunk-entry work chunks
    uint32_t *chunk_tile = nullptr;  // the tile of each work chunk (tiles + list_cap / kSplatChunk + 1)
    uint32_t *tile_list = nullptr;   // list_cap particle indices
    uint32_t list_cap = 0;
    unsigned long long *list_used = nullptr;  // entries reserved this step (64-bit: rejected reservations count too)
    uint8_t *accepted = nullptr;     // n: the sphere is in the tile lists
    uint2 *box = nullptr;            // n: screen box of an accepted sphere (x0 | x1 << 16, y0 | y1 << 16)
    float *near = nullptr;           // n: lower bound of the sphere's entry distances
    uint32_t *open_mask = nullptr;   // n: which of an accepted sphere's <= 32 box tiles it is listed in
    uint32_t *tile_max = nullptr;    // tiles: farthest depth bits of the phase-0 image
    uint32_t *big = nullptr;         // n: spheres rasterised one block each
    uint32_t *big_cnt = nullptr;
    void *alloc = nullptr;           // the one device allocation holding all of the above
    size_t alloc_bytes = 0;
};

// A texture object over a record array (raw 32-bit words): record e is
// texel e + off (the texture starts at the array's address rounded down to the
// device's texture alignment). t = 0: the array has no texture object.
struct RecTex {
    cudaTextureObject_t t = 0;
    uint32_t off = 0;
};

struct Buffers {
    float4 *state_x, *state_v;
    uint32_t *state_id;
    uint32_t *key, *slot;
    uint8_t *lvl;
    uint32_t *cnt, *start, *tile_sums, *tmp;
    float4 *recA, *recB, *xs32, *xt;
    uint32_t *id_s, *cell_s;
    uint8_t *lvl_s, *nbr_cnt;     // nbr_cnt and nbr: by list column (see partitioned())
    uint32_t *nbr;
    uint8_t *prev_cnt;            // neighbour count of each state slot in the last step
    RecTex texXt;                 // texture object over xt (the velocity pass), t = 0: none
    float *rho;
    float *lodd;                   // DTVS distance behind the visible surface, state order (-1: outside the view)
    uint32_t *act, *lvl_hist, *lvl_off, *lvl_count;
    unsigned long long *counters;  // kCounterSlots: see kDiagCounterSlot, kIterTotalSlot
    uint32_t *drange;              // ~(float bits) of d_min (scenes entries), then float bits of d_max
    const SceneGeom *geo;          // per scene
    const uint16_t *sid;           // scene of each particle slot (constant)
    uint32_t *err;                 // device error word (kErr* bits) of the step
    uint32_t *err_scene;           // the same bits per scene (a batch fails only the scenes that set them)
    uint32_t *dbg;                 // debug-build checks: first failure's code and index, plant request
    DynParams *dyn;                // per scene
    float4 *snap_x, *snap_v;       // state snapshot for the autotuner
    uint32_t *snap_id;
    float *stage_f;                // 3n floats readback staging
    uint8_t *stage_u8;             // n bytes readback staging
    float4 *dbg4;                  // n float4 debug staging
    double *partials;              // diagnostic partial sums
    double *dstats;                // 4 doubles
};

// Launch configuration of the solver passes, picked per scene by the autotuner.
struct Tune {
    int block = 256;              // threads per block of the lambda / delta-p kernels (128 or 256)
    float mask_threshold = 2.0f;  // iterate masked over all particles when |P_l| >= threshold * n
};

struct TimedLaunch {
    uint32_t stage;
    cudaEvent_t a, b;
};

}  // namespace apbf

struct apbf_scene {
    int device = 0;
    apbf::StepConst sc{};
    std::vector<apbf::SceneGeom> geo;  // host copy of the per-scene geometry
    apbf::Buffers b{};
    cudaStream_t stream = nullptr;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    bool own_arena = false;
    uint32_t flags = 0;
    int sms = 0;
    int grid_iter = 0;  // persistent grid of the iteration kernels
    apbf::Tune tune;
    apbf::ViewConst view;  // DTVS camera image (single scenes)
    bool view_set = false;
    // dynamic parameters, one per scene
    std::vector<apbf::DynParams> dyn;
    std::vector<float> grid_hi3;             // per scene static grid upper bounds (3 each)
    bool dyn_dirty = true;
    apbf::DynParams *dyn_pinned = nullptr;  // ring of 16 pinned upload slots of dyn_cap entries each
    uint32_t dyn_cap = 1;                   // scenes the arena was carved for
    cudaEvent_t dyn_ev[16] = {};
    int dyn_slot = 0;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t capture_stream = nullptr;
    // state
    bool stepped = false;
    int cur_buf = 0;  // debug: 0 = recA, 1 = recB holds the current positions
    bool lists_by_slot = true;  // the neighbour lists were last written by sorted slot (density diagnostic)
    apbf_status sticky = APBF_OK;
    std::string msg;
    // timing
    bool timing = false;
    std::vector<apbf::TimedLaunch> timed;
    std::vector<cudaEvent_t> ev_pool;
    double stage_ms[APBF_STAGE_COUNT] = {};
    uint64_t stage_launches[APBF_STAGE_COUNT] = {};
    // asynchronous position readback: the copy runs on its own stream while
    // the next step computes; copy_ev marks the end of the last such copy
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t unperm_ev = nullptr, copy_ev = nullptr;
    bool copy_pending = false;
    // host pinned scratch for small readbacks
    void *pinned_small = nullptr;
};

namespace apbf {

// A step partitions the particles by level (the active list act) when the LOD
// spans more than one level; the neighbour lists are then stored by
// active-list position (column t holds the particle act[t]), otherwise by
// sorted slot.
inline bool partitioned(const StepConst &sc) { return sc.lod_mode != APBF_LOD_FIXED && sc.K > 1; }
// Bytes of the region zeroed at the start of every step: the level counts per
// tile, the distance range and the step's counters (carved in this order).
inline size_t step_zero_bytes(const Buffers &b)
{
    return (size_t)((const char *)(b.counters + kDiagCounterSlot) - (const char *)b.lvl_hist);
}

// Kernel launchers (kernels.cu). Each returns cudaGetLastError().
cudaError_t launch_predict_hash(const StepConst &sc, const Buffers &b, cudaStream_t s, bool diag);
cudaError_t launch_scan(const StepConst &sc, const Buffers &b, cudaStream_t s);
cudaError_t launch_scatter(const StepConst &sc, const Buffers &b, cudaStream_t s);
cudaError_t launch_reorder(const StepConst &sc, const Buffers &b, cudaStream_t s, bool diag);
cudaError_t launch_neighbors(const StepConst &sc, const Buffers &b, cudaStream_t s, bool part);
cudaError_t launch_levels(const StepConst &sc, const Buffers &b, cudaStream_t s);
cudaError_t launch_lambda(const StepConst &sc, const Buffers &b, cudaStream_t s, uint32_t l, bool dense, int sms,
                          const Tune &tune);
cudaError_t launch_deltap(const StepConst &sc, const Buffers &b, cudaStream_t s, uint32_t l, bool dense, int sms,
                          const Tune &tune);
cudaError_t launch_finalize(const StepConst &sc, const Buffers &b, cudaStream_t s);
cudaError_t launch_prestab(const StepConst &sc, const Buffers &b, cudaStream_t s);
cudaError_t launch_dtvs(const StepConst &sc, const Buffers &b, const ViewConst &v, int sms, cudaStream_t s);
cudaError_t launch_unpermute(const StepConst &sc, const Buffers &b, cudaStream_t s, uint32_t what);
cudaError_t launch_density(const StepConst &sc, const Buffers &b, cudaStream_t s, int *nblocks);
cudaError_t launch_debug_xstar(const StepConst &sc, const Buffers &b, const float4 *rec, cudaStream_t s);
cudaError_t launch_debug_lambda(const StepConst &sc, const Buffers &b, const float4 *rec, cudaStream_t s);
cudaError_t launch_fixed_levels(const StepConst &sc, const Buffers &b, cudaStream_t s);
int iteration_grid(int sms);

// Host helpers shared by the scene / batch entry points and the server (apbf_capi.cu).
std::string derive(const apbf_scene_desc *d, StepConst &sc, apbf_status &st);
// Exponent e of the fixed-point unit 2^e of a scene with this h whose grid is
// short enough: the smallest e with 2^(e + 22) >= h.
int fx_exponent_for_h(float h);
bool same_physics(const apbf_scene_desc &a, const apbf_scene_desc &d);
size_t carve(const StepConst &sc, char *base, Buffers &b);
apbf_status alloc_scene(const StepConst &cap, uint32_t flags, void *cuda_stream, void *device_arena,
                        size_t arena_bytes, apbf_scene **out, std::string &msg);
void drop_graph(apbf_scene *s);
void set_last_error_message(const std::string &m);

}  // namespace apbf
