// Serving loop of include/apbf.h (apbf_server_*): independent scenes arrive
// over time, wait in a FIFO queue, are admitted into one resident pool while
// its capacity (sized from an HBM budget) has room, and every resident scene
// advances one step of Fig. 7 per tick, all of them in one batched step.
// Finished scenes are read back to the caller's buffers and leave the pool.
//
// The pool is a batch scene whose arena is carved for the capacity; a
// membership change rewrites its scene table and moves the surviving scenes'
// state down to close the gaps. A scene's arithmetic and its particles'
// relative order do not depend on its place in the pool, so every scene
// evolves bit-identically to the same scene stepped alone.
#include <cmath>
#include <cstring>
#include <deque>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "apbf_internal.h"

using namespace apbf;

namespace {

constexpr uint32_t kMaxSlots = kMaxParticles - 1u;

struct Request {
    uint64_t ticket = 0;
    apbf_scene_desc desc{};
    std::vector<float> pos, vel;  // released once uploaded
    StepConst geo{};              // the scene's own derived grid
    float eye[3] = {};
    uint32_t steps = 0, done = 0;
    float *pos_out = nullptr, *vel_out = nullptr;
    std::vector<Obstacle> obst;  // the scene's obstacles
    uint32_t state = APBF_REQ_QUEUED;
    apbf_status status = APBF_OK;  // why a failed request failed
    uint64_t submit_tick = 0, admit_tick = 0, done_tick = 0;
    uint32_t p0 = 0, cell_base = 0;  // place in the pool while resident
};

struct MoveSeg {
    uint32_t new_p0, old_p0, n, pad;
};

// Moves each surviving scene's state from its old slot range to its new one
// (into the other state buffer), re-basing the scene's global particle ids.
__global__ void move_kernel(const float4 *__restrict__ x0, const float4 *__restrict__ v0,
                            const uint32_t *__restrict__ id0, float4 *__restrict__ x1, float4 *__restrict__ v1,
                            uint32_t *__restrict__ id1, const MoveSeg *__restrict__ seg, uint32_t nseg, uint32_t n)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n)
        return;
    uint32_t lo = 0, hi = nseg;  // seg[lo].new_p0 <= g < seg[hi].new_p0
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (seg[mid].new_p0 <= g)
            lo = mid;
        else
            hi = mid;
    }
    const MoveSeg s = seg[lo];
    const uint32_t src = s.old_p0 + (g - s.new_p0);
    x1[g] = x0[src];
    v1[g] = v0[src];
    id1[g] = id0[src] - s.old_p0 + s.new_p0;
}

// Expands uploaded xyz triples of slots [g0, g1) to float4 state entries; with
// ids, a new scene's particles start in id order (global id = slot).
__global__ void place_kernel(const float *__restrict__ stage, float4 *__restrict__ dst, uint32_t *__restrict__ ids,
                             uint32_t g0, uint32_t g1)
{
    const uint32_t g = g0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= g1)
        return;
    dst[g] = make_float4(stage[3 * (size_t)g], stage[3 * (size_t)g + 1], stage[3 * (size_t)g + 2], 0.0f);
    if (ids)
        ids[g] = g;
}

// Scene index of every particle slot from the scene table's first slots.
__global__ void sid_kernel(const SceneGeom *__restrict__ geo, uint32_t scenes, uint16_t *__restrict__ sid, uint32_t n)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n)
        return;
    uint32_t lo = 0, hi = scenes;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (geo[mid].p0 <= g)
            lo = mid;
        else
            hi = mid;
    }
    sid[g] = (uint16_t)lo;
}

uint32_t blocks_of(uint32_t n) { return (n + kBlock - 1) / kBlock; }

// Pool capacity: `n` particles, `cells` cells and `scenes` scenes with the
// physics of `phys` (already derived).
StepConst capacity(const StepConst &phys, uint32_t n, uint32_t cells, uint32_t scenes)
{
    StepConst c = phys;
    c.n = n;
    c.ncell = cells;
    c.scenes = scenes;
    c.level_tiles = level_tile_count(n);
    return c;
}

size_t pool_bytes(const StepConst &cap)
{
    Buffers b{};
    return carve(cap, nullptr, b);
}

// Resolves the capacities of a server description; returns a message or "".
std::string resolve(const apbf_server_desc *d, StepConst &phys, StepConst &cap, apbf_status &st)
{
    st = APBF_ERR_INVALID_ARG;
    if (!d || !d->physics)
        return "desc or desc->physics is NULL";
    apbf_scene_desc p = *d->physics;
    p.n = 0;  // particles, grid and box of the physics description are not used
    p.pos = nullptr;
    p.vel = nullptr;
    for (int a = 0; a < 3; ++a) {
        p.grid_lo[a] = 0.0f;
        p.grid_hi[a] = p.h;
        p.box_lo[a] = 0.0f;
        p.box_hi[a] = p.h;
    }
    std::string m = derive(&p, phys, st);
    if (st != APBF_OK)
        return "physics: " + m;
    if (p.lod_mode == APBF_LOD_DTVS) {
        st = APBF_ERR_NOT_SUPPORTED;
        return "the server steps batches; DTVS scenes are single scenes";
    }
    st = APBF_ERR_INVALID_ARG;
    const uint32_t scenes = d->max_scenes ? d->max_scenes : 4096u;
    if (scenes > 65535u)
        return "max_scenes must be <= 65535";
    if (d->max_particles > kMaxSlots)
        return "max_particles must be below 2^31 - 1";
    auto cells_for = [&](uint32_t n) -> uint32_t {
        if (d->max_cells)
            return d->max_cells;
        const uint64_t c = 4ull * n;
        return (uint32_t)(c < (1ull << 31) - 1 ? c : (1ull << 31) - 1);
    };
    if (d->max_cells >= (1u << 31))
        return "max_cells must be below 2^31";
    if (!std::isfinite(d->target_step_ms) || d->target_step_ms < 0.0)
        return "target_step_ms must be finite and >= 0";
    uint32_t n = d->max_particles;
    if (n == 0) {
        if (d->budget_bytes == 0)
            return "give max_particles or budget_bytes";
        // the largest particle capacity whose pool fits the budget
        uint32_t lo = 0, hi = kMaxSlots;
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo + 1) / 2;
            if (pool_bytes(capacity(phys, mid, cells_for(mid), scenes)) <= d->budget_bytes)
                lo = mid;
            else
                hi = mid - 1;
        }
        if (lo == 0) {
            st = APBF_ERR_OUT_OF_MEMORY;
            return "budget_bytes is too small for a single particle";
        }
        n = lo;
    }
    cap = capacity(phys, n, cells_for(n), scenes);
    if (d->budget_bytes && pool_bytes(cap) > d->budget_bytes) {
        st = APBF_ERR_OUT_OF_MEMORY;
        return "the pool for these capacities exceeds budget_bytes";
    }
    st = APBF_OK;
    return "";
}

}  // namespace

struct apbf_server {
    apbf_scene *pool = nullptr;
    StepConst cap{};
    apbf_scene_desc physics{};
    std::deque<Request *> queue;
    std::vector<Request *> resident;  // in pool order
    std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
    uint64_t next_ticket = 1;
    uint64_t tick = 0;
    uint32_t n_res = 0, c_res = 0;
    MoveSeg *d_seg = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool in_flight = false;
    // host pinned: the step's error word, the per-scene error words, the running particle-iterations
    uint32_t *h_err = nullptr;
    unsigned long long *h_iters = nullptr;
    unsigned long long total_iters = 0;
    // admission by step-latency target: measured device ms per particle-step (running average)
    double target_ms = 0.0, cost_ms = 2.0e-6;
    uint32_t n_stepped = 0;
    apbf_status sticky = APBF_OK;
    std::string msg;
};

namespace {

apbf_status sfail(apbf_server *sv, apbf_status st, const std::string &m)
{
    if (sv) {
        sv->msg = m;
        if (st == APBF_ERR_CUDA || st == APBF_ERR_NEIGHBOR_OVERFLOW || st == APBF_ERR_TIMEOUT)
            sv->sticky = st;
    } else {
        set_last_error_message(m);
    }
    return st;
}

#define SV_CUDA(sv, expr)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return sfail((sv), APBF_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// A failure of the pool scene: every resident request fails with it.
apbf_status pool_fail(apbf_server *sv, apbf_status st)
{
    for (Request *r : sv->resident) {
        r->state = APBF_REQ_FAILED;
        r->status = st;
        r->done_tick = sv->tick;
    }
    return sfail(sv, st, std::string("pool: ") + apbf_last_error(sv->pool));
}

// Reads the finished requests' state back into their buffers.
apbf_status read_back(apbf_server *sv, const std::vector<Request *> &fin)
{
    apbf_scene *s = sv->pool;
    for (uint32_t what = 0; what < 2; ++what) {
        bool any = false;
        for (Request *r : fin)
            any = any || (what == 0 ? r->pos_out : r->vel_out);
        if (!any)
            continue;
        SV_CUDA(sv, launch_unpermute(s->sc, s->b, s->stream, what));
        for (Request *r : fin) {
            float *dst = what == 0 ? r->pos_out : r->vel_out;
            if (dst)
                SV_CUDA(sv, cudaMemcpyAsync(dst, s->b.stage_f + 3 * (size_t)r->p0, 12 * (size_t)r->desc.n,
                                            cudaMemcpyDeviceToHost, s->stream));
        }
        SV_CUDA(sv, cudaStreamSynchronize(s->stream));
    }
    return APBF_OK;
}

// Rewrites the pool's scene table, per-scene parameters and step constants
// for the current residents, and invalidates the captured step.
apbf_status relayout(apbf_server *sv)
{
    apbf_scene *s = sv->pool;
    const uint32_t count = (uint32_t)sv->resident.size();
    s->geo.assign(count, SceneGeom{});
    s->dyn.assign(count, DynParams{});
    s->grid_hi3.assign(3 * (size_t)count, 0.0f);
    for (uint32_t k = 0; k < count; ++k) {
        const Request *r = sv->resident[k];
        SceneGeom &g = s->geo[k];
        for (int a = 0; a < 3; ++a) {
            g.glo[a] = r->geo.glo[a];
            s->grid_hi3[3 * k + a] = r->desc.grid_hi[a];
            s->dyn[k].box_lo[a] = r->desc.box_lo[a];
            s->dyn[k].box_hi[a] = r->desc.box_hi[a];
            s->dyn[k].eye[a] = r->eye[a];
            s->dyn[k].dir[a] = a == 0 ? 1.0f : 0.0f;
        }
        s->dyn[k].n_obst = (uint32_t)r->obst.size();
        for (size_t o = 0; o < r->obst.size(); ++o)
            s->dyn[k].obst[o] = r->obst[o];
        g.nx = r->geo.nx;
        g.ny = r->geo.ny;
        g.nz = r->geo.nz;
        g.cell_base = r->cell_base;
        g.p0 = r->p0;
        g.n = r->desc.n;
        s->dyn[k].auto_range = 1;
    }
    StepConst &sc = s->sc;
    sc.n = sv->n_res;
    sc.ncell = sv->c_res;
    sc.scenes = count ? count : 1;
    sc.level_tiles = level_tile_count(sc.n);
    if (count == 1) {  // the single-scene kernels read the grid from the step constants
        const StepConst &g = sv->resident[0]->geo;
        for (int a = 0; a < 3; ++a)
            sc.glo[a] = g.glo[a];
        sc.nx = g.nx;
        sc.ny = g.ny;
        sc.nz = g.nz;
    }
    if (count) {
        SV_CUDA(sv, cudaMemcpyAsync((void *)s->b.geo, s->geo.data(), sizeof(SceneGeom) * count,
                                    cudaMemcpyHostToDevice, s->stream));
        if (sc.n)
            sid_kernel<<<blocks_of(sc.n), kBlock, 0, s->stream>>>(s->b.geo, count, (uint16_t *)s->b.sid, sc.n);
        SV_CUDA(sv, cudaGetLastError());
    }
    s->dyn_dirty = true;
    drop_graph(s);
    return APBF_OK;
}

apbf_status tick_impl(apbf_server *sv, apbf_tick_info *info)
{
    apbf_scene *s = sv->pool;
    std::memset(info, 0, sizeof(*info));
    info->tick = sv->tick;
    // 1. the previous tick's step
    if (sv->in_flight) {
        SV_CUDA(sv, cudaEventSynchronize(sv->ev1));
        float ms = 0.0f;
        SV_CUDA(sv, cudaEventElapsedTime(&ms, sv->ev0, sv->ev1));
        info->prev_step_ms = ms;
        sv->in_flight = false;
        if (sv->n_stepped >= 262144u) {
            const double c = (double)ms / sv->n_stepped;
            sv->cost_ms = 0.7 * sv->cost_ms + 0.3 * c;
        }
        // a neighbour overflow fails only the scenes that had it: their words are
        // read, those requests retire as failed, and the words are cleared, so the
        // pool itself goes on (any other device error still fails the pool)
        const uint32_t count = (uint32_t)sv->resident.size();
        SV_CUDA(sv, cudaMemcpyAsync(sv->h_err, s->b.err, 4, cudaMemcpyDeviceToHost, s->stream));
        SV_CUDA(sv, cudaMemcpyAsync(sv->h_err + 1, s->b.err_scene, 4 * (size_t)count, cudaMemcpyDeviceToHost,
                                    s->stream));
        SV_CUDA(sv, cudaMemcpyAsync(sv->h_iters, s->b.counters + kIterTotalSlot, 8, cudaMemcpyDeviceToHost,
                                    s->stream));
        SV_CUDA(sv, cudaStreamSynchronize(s->stream));
        sv->total_iters = *sv->h_iters;
        if (sv->h_err[0] == kErrNeighborOverflow) {
            for (uint32_t k = 0; k < count; ++k)
                if (sv->h_err[1 + k] & kErrNeighborOverflow) {
                    Request *r = sv->resident[k];
                    r->state = APBF_REQ_FAILED;
                    r->status = APBF_ERR_NEIGHBOR_OVERFLOW;
                    r->done_tick = sv->tick;
                }
            SV_CUDA(sv, cudaMemsetAsync(s->b.err, 0, 4, s->stream));
            SV_CUDA(sv, cudaMemsetAsync(s->b.err_scene, 0, 4 * (size_t)count, s->stream));
        }
        apbf_status st = apbf_sync(s);
        if (st != APBF_OK)
            return pool_fail(sv, st);
    }
    info->total_particle_iterations = sv->total_iters;
    // 2. retire finished scenes
    std::vector<Request *> fin, kept;
    uint32_t failed = 0;
    for (Request *r : sv->resident) {
        if (r->state == APBF_REQ_FAILED)
            ++failed;
        else
            (r->done >= r->steps ? fin : kept).push_back(r);
    }
    bool changed = false;
    if (!fin.empty() || failed) {
        apbf_status st = read_back(sv, fin);
        if (st != APBF_OK)
            return st;
        for (Request *r : fin) {
            r->state = APBF_REQ_DONE;
            r->done_tick = sv->tick;
        }
        info->completed = (uint32_t)fin.size();
        info->failed = failed;
        // 3. close the gaps: survivors keep their order and move down
        std::vector<MoveSeg> seg;
        uint32_t p = 0, c = 0;
        bool moved = false;
        for (Request *r : kept) {
            seg.push_back(MoveSeg{p, r->p0, r->desc.n, 0u});
            moved = moved || r->p0 != p;
            r->p0 = p;
            r->cell_base = c;
            p += r->desc.n;
            c += r->geo.ncell;
        }
        if (moved) {
            Buffers &b = s->b;
            SV_CUDA(sv, cudaMemcpyAsync(sv->d_seg, seg.data(), sizeof(MoveSeg) * seg.size(), cudaMemcpyHostToDevice,
                                        s->stream));
            move_kernel<<<blocks_of(p), kBlock, 0, s->stream>>>(b.state_x, b.state_v, b.state_id, b.snap_x, b.snap_v,
                                                                 b.snap_id, sv->d_seg, (uint32_t)seg.size(), p);
            SV_CUDA(sv, cudaGetLastError());
            std::swap(b.state_x, b.snap_x);
            std::swap(b.state_v, b.snap_v);
            std::swap(b.state_id, b.snap_id);
        }
        sv->resident = kept;
        sv->n_res = p;
        sv->c_res = c;
        changed = true;
    }
    // 4. admit from the queue in arrival order while the pool has room
    const uint32_t first_new = (uint32_t)sv->resident.size();
    const uint32_t n_before = sv->n_res;
    uint32_t limit = sv->cap.n;
    if (sv->target_ms > 0.0) {
        const double l = 0.9 * sv->target_ms / sv->cost_ms;
        limit = l < (double)sv->cap.n ? (uint32_t)l : sv->cap.n;
    }
    info->particle_limit = limit;
    while (!sv->queue.empty()) {
        Request *r = sv->queue.front();
        if ((uint64_t)sv->n_res + r->desc.n > sv->cap.n || (uint64_t)sv->c_res + r->geo.ncell > sv->cap.ncell ||
            sv->resident.size() + 1 > sv->cap.scenes)
            break;
        if (!sv->resident.empty() && (uint64_t)sv->n_res + r->desc.n > limit)
            break;  // the step would exceed the latency target: wait (arrival order is kept)
        sv->queue.pop_front();
        r->p0 = sv->n_res;
        r->cell_base = sv->c_res;
        r->state = APBF_REQ_RESIDENT;
        r->admit_tick = sv->tick;
        sv->n_res += r->desc.n;
        sv->c_res += r->geo.ncell;
        sv->resident.push_back(r);
        info->admitted += 1;
        changed = true;
    }
    if (info->admitted) {
        // upload the new scenes' positions, then velocities, through the readback staging buffer
        Buffers &b = s->b;
        for (uint32_t what = 0; what < 2; ++what) {
            for (uint32_t k = first_new; k < sv->resident.size(); ++k) {
                Request *r = sv->resident[k];
                float *dst = b.stage_f + 3 * (size_t)r->p0;
                const std::vector<float> &src = what == 0 ? r->pos : r->vel;
                if (src.empty())
                    SV_CUDA(sv, cudaMemsetAsync(dst, 0, 12 * (size_t)r->desc.n, s->stream));
                else
                    SV_CUDA(sv, cudaMemcpyAsync(dst, src.data(), 12 * (size_t)r->desc.n, cudaMemcpyHostToDevice,
                                                s->stream));
            }
            place_kernel<<<blocks_of(sv->n_res - n_before), kBlock, 0, s->stream>>>(
                b.stage_f, what == 0 ? b.state_x : b.state_v, what == 0 ? b.state_id : nullptr, n_before, sv->n_res);
            SV_CUDA(sv, cudaGetLastError());
        }
        SV_CUDA(sv, cudaStreamSynchronize(s->stream));  // the host copies are read before they are released
        for (uint32_t k = first_new; k < sv->resident.size(); ++k) {
            std::vector<float>().swap(sv->resident[k]->pos);
            std::vector<float>().swap(sv->resident[k]->vel);
        }
    }
    if (changed) {
        apbf_status st = relayout(sv);
        if (st != APBF_OK)
            return st;
    }
    // 5. one step of every resident scene
    info->resident_scenes = (uint32_t)sv->resident.size();
    info->resident_particles = sv->n_res;
    info->queued = (uint32_t)sv->queue.size();
    if (!sv->resident.empty()) {
        SV_CUDA(sv, cudaEventRecord(sv->ev0, s->stream));
        sv->n_stepped = sv->n_res;
        apbf_status st = apbf_step(s, 1);
        if (st != APBF_OK)
            return pool_fail(sv, st);
        SV_CUDA(sv, cudaEventRecord(sv->ev1, s->stream));
        sv->in_flight = true;
        for (Request *r : sv->resident)
            r->done += 1;
    }
    sv->tick += 1;
    return APBF_OK;
}

}  // namespace

extern "C" {

APBF_API apbf_status apbf_server_bytes(const apbf_server_desc *desc, size_t *bytes, uint32_t *max_particles,
                                       uint32_t *max_cells)
{
    StepConst phys, cap;
    apbf_status st;
    std::string m = resolve(desc, phys, cap, st);
    if (st != APBF_OK)
        return sfail(nullptr, st, m);
    if (bytes)
        *bytes = pool_bytes(cap);
    if (max_particles)
        *max_particles = cap.n;
    if (max_cells)
        *max_cells = cap.ncell;
    return APBF_OK;
}

APBF_API apbf_status apbf_server_create(const apbf_server_desc *desc, void *cuda_stream, apbf_server **out)
{
    if (!out)
        return sfail(nullptr, APBF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    StepConst phys, cap;
    apbf_status st;
    std::string m = resolve(desc, phys, cap, st);
    if (st != APBF_OK)
        return sfail(nullptr, st, m);
    std::unique_ptr<apbf_server> sv(new (std::nothrow) apbf_server());
    if (!sv)
        return sfail(nullptr, APBF_ERR_OUT_OF_MEMORY, "host allocation failed");
    sv->cap = cap;
    sv->target_ms = desc->target_step_ms;
    sv->physics = *desc->physics;
    sv->physics.pos = nullptr;
    sv->physics.vel = nullptr;
    st = alloc_scene(cap, desc->physics->flags, cuda_stream, nullptr, 0, &sv->pool, m);
    if (st != APBF_OK)
        return sfail(nullptr, st, m);
    cudaError_t e;
    if ((e = cudaMalloc(&sv->d_seg, sizeof(MoveSeg) * cap.scenes)) != cudaSuccess ||
        (e = cudaEventCreate(&sv->ev0)) != cudaSuccess || (e = cudaEventCreate(&sv->ev1)) != cudaSuccess ||
        (e = cudaMallocHost(&sv->h_err, 4 * (size_t)(cap.scenes + 1))) != cudaSuccess ||
        (e = cudaMallocHost(&sv->h_iters, 8)) != cudaSuccess ||
        (e = cudaStreamSynchronize(sv->pool->stream)) != cudaSuccess) {
        cudaGetLastError();
        apbf_server_destroy(sv.release());
        return sfail(nullptr, APBF_ERR_CUDA, std::string("server setup: ") + cudaGetErrorString(e));
    }
    relayout(sv.get());
    *out = sv.release();
    return APBF_OK;
}

APBF_API apbf_status apbf_server_submit(apbf_server *sv, const apbf_request *req, uint64_t *ticket)
{
    if (!sv)
        return APBF_ERR_INVALID_ARG;
    if (sv->sticky != APBF_OK)
        return sv->sticky;
    if (!req || !req->scene || !ticket)
        return sfail(sv, APBF_ERR_INVALID_ARG, "req, req->scene or ticket is NULL");
    const apbf_scene_desc *d = req->scene;
    if (d->n == 0 || req->steps == 0)
        return sfail(sv, APBF_ERR_INVALID_ARG, "a request needs n >= 1 and steps >= 1");
    if (!std::isfinite(req->eye[0]) || !std::isfinite(req->eye[1]) || !std::isfinite(req->eye[2]))
        return sfail(sv, APBF_ERR_INVALID_ARG, "eye must be finite");
    if (!same_physics(sv->physics, *d))
        return sfail(sv, APBF_ERR_INVALID_ARG, "the scene's physics differs from the server's");
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r)
        return sfail(sv, APBF_ERR_OUT_OF_MEMORY, "host allocation failed");
    apbf_status st;
    std::string m = derive(d, r->geo, st);
    if (st != APBF_OK)
        return sfail(sv, st, m);
    if (d->n > sv->cap.n || r->geo.ncell > sv->cap.ncell)
        return sfail(sv, APBF_ERR_INVALID_ARG, "the scene alone exceeds the server's particle or cell capacity");
    if (r->geo.fx_e != fx_exponent_for_h(d->h))
        return sfail(sv, APBF_ERR_NOT_SUPPORTED, "the scene's grid spans 8e8 or more fixed-point units on an axis; "
                                                 "such scenes step alone, not in a pool");
    const size_t n3 = 3 * (size_t)d->n;
    for (size_t i = 0; i < n3; ++i)
        if (!std::isfinite(d->pos[i]) || (d->vel && !std::isfinite(d->vel[i])))
            return sfail(sv, APBF_ERR_INVALID_ARG, "positions and velocities must be finite");
    for (uint32_t i = 0; i < d->n; ++i)
        for (int a = 0; a < 3; ++a)
            if (!(d->pos[3 * i + a] >= d->grid_lo[a] && d->pos[3 * i + a] <= d->grid_hi[a]))
                return sfail(sv, APBF_ERR_INVALID_ARG, "particle " + std::to_string(i) + " lies outside the grid");
    r->pos.assign(d->pos, d->pos + n3);
    if (d->vel)
        r->vel.assign(d->vel, d->vel + n3);
    r->desc = *d;
    r->desc.pos = nullptr;
    r->desc.vel = nullptr;
    for (int a = 0; a < 3; ++a)
        r->eye[a] = req->eye[a];
    if (req->n_obstacles > APBF_MAX_OBSTACLES || (req->n_obstacles && !req->obstacles))
        return sfail(sv, APBF_ERR_INVALID_ARG, "need n_obstacles <= APBF_MAX_OBSTACLES and a non-NULL array");
    for (uint32_t k = 0; k < req->n_obstacles; ++k) {
        const apbf_obstacle &o = req->obstacles[k];
        bool ok = std::isfinite(o.a[0]) && std::isfinite(o.a[1]) && std::isfinite(o.a[2]) && std::isfinite(o.b[0]) &&
                  std::isfinite(o.b[1]) && std::isfinite(o.b[2]);
        if (o.kind == APBF_OBSTACLE_SPHERE)
            ok = ok && o.b[0] > 0.0f;
        else if (o.kind == APBF_OBSTACLE_BOX)
            ok = ok && o.a[0] < o.b[0] && o.a[1] < o.b[1] && o.a[2] < o.b[2];
        else if (o.kind == APBF_OBSTACLE_CONE)
            ok = ok && o.b[0] > 0.0f && o.b[1] > 0.0f;
        else
            ok = false;
        if (!ok)
            return sfail(sv, APBF_ERR_INVALID_ARG, "obstacle " + std::to_string(k) + ": unknown kind or bad size");
        Obstacle q{};
        q.kind = o.kind;
        for (int a = 0; a < 3; ++a) {
            q.a[a] = o.a[a];
            q.b[a] = o.b[a];
        }
        r->obst.push_back(q);
    }
    r->steps = req->steps;
    r->pos_out = req->pos_out;
    r->vel_out = req->vel_out;
    r->ticket = sv->next_ticket++;
    r->submit_tick = sv->tick;
    *ticket = r->ticket;
    sv->queue.push_back(r.get());
    sv->all.emplace(r->ticket, std::move(r));
    return APBF_OK;
}

APBF_API apbf_status apbf_server_tick(apbf_server *sv, apbf_tick_info *info)
{
    if (!sv)
        return APBF_ERR_INVALID_ARG;
    if (sv->sticky != APBF_OK)
        return sv->sticky;
    apbf_tick_info local;
    return tick_impl(sv, info ? info : &local);
}

APBF_API apbf_status apbf_server_query(apbf_server *sv, uint64_t ticket, apbf_request_info *info)
{
    if (!sv || !info)
        return APBF_ERR_INVALID_ARG;
    auto it = sv->all.find(ticket);
    if (it == sv->all.end())
        return sfail(sv, APBF_ERR_INVALID_ARG, "unknown ticket");
    const Request &r = *it->second;
    info->state = r.state;
    info->steps_done = r.state == APBF_REQ_QUEUED ? 0u : (r.done < r.steps ? r.done : r.steps);
    info->n = r.desc.n;
    info->steps = r.steps;
    info->submit_tick = r.submit_tick;
    info->admit_tick = r.admit_tick;
    info->done_tick = r.done_tick;
    info->status = r.status;
    info->pad = 0;
    return APBF_OK;
}

APBF_API const char *apbf_server_last_error(const apbf_server *sv)
{
    return sv ? sv->msg.c_str() : apbf_last_error(nullptr);
}

APBF_API void apbf_server_destroy(apbf_server *sv)
{
    if (!sv)
        return;
    if (sv->pool)
        apbf_destroy_scene(sv->pool);  // synchronises the pool's stream
    if (sv->d_seg)
        cudaFree(sv->d_seg);
    if (sv->ev0)
        cudaEventDestroy(sv->ev0);
    if (sv->ev1)
        cudaEventDestroy(sv->ev1);
    if (sv->h_err)
        cudaFreeHost(sv->h_err);
    if (sv->h_iters)
        cudaFreeHost(sv->h_iters);
    delete sv;
}

}  // extern "C"
