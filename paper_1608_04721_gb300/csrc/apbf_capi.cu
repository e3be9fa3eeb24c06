// Host side of the C ABI declared in include/apbf.h: validation, the device
// arena, step orchestration (eager launches or a captured CUDA graph),
// readback, diagnostics, timing and test-only exports.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "apbf_internal.h"

using namespace apbf;

namespace {

thread_local std::string g_create_error;

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

apbf_status fail(apbf_scene *s, apbf_status st, const std::string &m)
{
    if (s) {
        s->msg = m;
        if (st == APBF_ERR_CUDA || st == APBF_ERR_NEIGHBOR_OVERFLOW || st == APBF_ERR_TIMEOUT ||
            st == APBF_ERR_CHECK_FAILED)
            s->sticky = st;
    } else {
        g_create_error = m;
    }
    return st;
}

apbf_status cuda_fail(apbf_scene *s, cudaError_t e, const char *where)
{
    return fail(s, APBF_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define APBF_CUDA(s, expr)                                \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess)                            \
            return cuda_fail((s), e_, #expr);             \
    } while (0)

bool finite3(const float *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

}  // namespace

namespace apbf {
int fx_exponent_for_h(float h)
{
    int e2;
    const double f = std::frexp((double)h, &e2);  // h = f 2^e2, f in [0.5, 1)
    return (f == 0.5 ? e2 - 1 : e2) - 22;          // ceil(log2 h) - 22
}

// Derived constants of a description; returns an error message or "".
std::string derive(const apbf_scene_desc *d, StepConst &sc, apbf_status &st)
{
    st = APBF_ERR_INVALID_ARG;
    if (!d)
        return "desc is NULL";
    if (d->n >= kMaxParticles)
        return "n must be below 2^31 - 1";
    if (d->n > 0 && !d->pos)
        return "pos is NULL";
    if (!(d->h > 0.0f) || !std::isfinite(d->h))
        return "h must be positive and finite";
    if (!(d->dt > 0.0f) || !std::isfinite(d->dt))
        return "dt must be positive and finite";
    if (!(d->mass > 0.0f) || !std::isfinite(d->mass))
        return "mass must be positive and finite";
    if (!(d->rho0 > 0.0f) || !std::isfinite(d->rho0))
        return "rho0 must be positive and finite";
    if (!(d->eps >= 0.0f) || !std::isfinite(d->eps))
        return "eps must be >= 0 and finite";
    if (!std::isfinite(d->scorr_k) || !(d->scorr_dq >= 0.0f) || !(d->scorr_dq < d->h) || d->scorr_n > 16)
        return "tensile term needs finite k, 0 <= dq < h and n <= 16";
    if (!std::isfinite(d->xsph_c) || !finite3(d->gravity))
        return "xsph_c and gravity must be finite";
    if (d->n_min < 1 || d->n_max < d->n_min || d->n_max > 255)
        return "need 1 <= n_min <= n_max <= 255";
    if (d->lod_mode != APBF_LOD_FIXED && d->lod_mode != APBF_LOD_DTC && d->lod_mode != APBF_LOD_DTVS)
        return "unknown lod_mode";
    if (d->stabil_s > d->n_max || d->stabil_iters > 64)
        return "pre-stabilisation needs S <= n_max and stabil_iters <= 64";
    if (d->max_neighbors > 255)
        return "max_neighbors must be <= 255";
    if (d->flags & ~APBF_FLAG_NO_GRAPH)
        return "unknown flag";
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(d->grid_lo[a]) || !std::isfinite(d->grid_hi[a]) || !std::isfinite(d->box_lo[a]) ||
            !std::isfinite(d->box_hi[a]))
            return "grid and box bounds must be finite";
        if (!(d->grid_lo[a] <= d->box_lo[a] && d->box_lo[a] < d->box_hi[a] && d->box_hi[a] <= d->grid_hi[a]))
            return "need grid_lo <= box_lo < box_hi <= grid_hi on every axis";
    }
    sc = StepConst{};
    sc.n = d->n;
    sc.inv_h = 1.0f / d->h;
    int dims[3];
    for (int a = 0; a < 3; ++a) {
        volatile float ext = d->grid_hi[a] - d->grid_lo[a];
        volatile float t = ext * sc.inv_h;
        double fl = std::floor((double)t);
        if (fl > 4096.0)
            return "grid too large for the cell packing";
        dims[a] = (int)fl + 1;
        sc.glo[a] = d->grid_lo[a];
    }
    if (dims[0] > 2047 || dims[1] > 2047 || dims[2] > 1023)
        return "grid must have at most 2047 x 2047 x 1023 cells";
    uint64_t ncell = (uint64_t)dims[0] * dims[1] * dims[2];
    if (ncell >= (1ull << 31))
        return "grid has too many cells";
    sc.nx = dims[0];
    sc.ny = dims[1];
    sc.nz = dims[2];
    sc.ncell = (uint32_t)ncell;
    sc.h = d->h;
    sc.h2 = d->h * d->h;
    sc.dt = d->dt;
    sc.inv_dt = (float)(1.0 / (double)d->dt);
    for (int a = 0; a < 3; ++a)
        sc.g[a] = d->gravity[a];
    // fixed-point unit: the smallest power of two u with 2^22 u >= h whose grid
    // spans fewer than kFxSpan units (a longer grid takes a coarser unit)
    sc.fx_e = fx_exponent_for_h(d->h);
    for (;;) {
        double span = 0.0;
        for (int a = 0; a < 3; ++a)
            span = std::max(span, std::ldexp((double)d->grid_hi[a] - (double)d->grid_lo[a], -sc.fx_e) + 2.0);
        if (span < kFxSpan)
            break;
        ++sc.fx_e;
    }
    sc.fx_u = (float)std::ldexp(1.0, sc.fx_e);
    sc.fx_inv_u = (float)std::ldexp(1.0, -sc.fx_e);
    sc.fx_off = (float)std::ldexp(-1.5, 23 + sc.fx_e);
    const double PI = 3.14159265358979323846;
    const double h = d->h, m = d->mass, rho0 = d->rho0, w = 1.0 / m;
    const double poly6 = 315.0 / (64.0 * PI * std::pow(h, 9));
    const double spiky = 45.0 / (PI * std::pow(h, 6));
    const double h2 = h * h;
    sc.mass_poly6 = (float)(m * poly6);
    sc.h6 = (float)(h2 * h2 * h2);
    sc.inv_rho0 = (float)(1.0 / rho0);
    sc.c_lam = (float)(w * (m * spiky / rho0) * (m * spiky / rho0));
    sc.eps = d->eps;
    sc.c_dp = (float)(-(w * m / rho0) * spiky);
    sc.c_dpu = (float)std::ldexp((double)sc.c_dp, -sc.fx_e);
    sc.v_scale = (float)((double)sc.fx_u / (double)d->dt);
    const double dq = d->scorr_dq;
    sc.inv_wdq = (float)(1.0 / (h2 - dq * dq));
    sc.neg_k = -d->scorr_k;
    sc.scorr_n = d->scorr_n;
    sc.c_xsph = (float)((double)d->xsph_c * (m / rho0) * poly6);
    sc.n_min = d->lod_mode == APBF_LOD_FIXED ? d->n_max : d->n_min;
    sc.dtvs_outside = sc.n_min;
    sc.n_max = d->n_max;
    sc.K = sc.n_max - sc.n_min + 1;
    sc.lod_mode = d->lod_mode;
    sc.max_nbr = d->max_neighbors ? d->max_neighbors : kDefaultMaxNeighbors;
    sc.level_tiles = level_tile_count(d->n);
    sc.rho0 = d->rho0;
    sc.stabil_s = d->stabil_s;
    sc.stabil_iters = d->stabil_iters;
    sc.scenes = 1;
    st = APBF_OK;
    return "";
}

bool same_physics(const apbf_scene_desc &a, const apbf_scene_desc &d)
{
    bool same = a.h == d.h && a.dt == d.dt && a.mass == d.mass && a.rho0 == d.rho0 && a.eps == d.eps &&
                a.scorr_k == d.scorr_k && a.scorr_dq == d.scorr_dq && a.scorr_n == d.scorr_n &&
                a.xsph_c == d.xsph_c && a.n_min == d.n_min && a.n_max == d.n_max && a.lod_mode == d.lod_mode &&
                a.stabil_s == d.stabil_s && a.stabil_iters == d.stabil_iters && a.max_neighbors == d.max_neighbors &&
                a.flags == d.flags;
    for (int ax = 0; ax < 3; ++ax)
        same = same && a.gravity[ax] == d.gravity[ax];
    return same;
}
}  // namespace apbf

namespace {
// Validation and derived constants of a batch: every scene is validated on
// its own; the physics (everything but particles, grid and box) must match
// scene 0; the scenes' particles and cells are concatenated.
std::string derive_batch(const apbf_scene_desc *descs, uint32_t count, StepConst &sc, std::vector<SceneGeom> &geo,
                         apbf_status &st)
{
    st = APBF_ERR_INVALID_ARG;
    if (!descs || count == 0)
        return "descs is NULL or count is 0";
    if (count > 65535)
        return "at most 65535 scenes per batch";
    if (count > 1 && descs[0].lod_mode == APBF_LOD_DTVS) {
        st = APBF_ERR_NOT_SUPPORTED;
        return "the DTVS model renders one camera image per scene; batches of DTVS scenes are not built";
    }
    geo.assign(count, SceneGeom{});
    uint64_t n_total = 0, c_total = 0;
    for (uint32_t k = 0; k < count; ++k) {
        StepConst sk;
        std::string m = derive(descs + k, sk, st);
        if (st != APBF_OK)
            return "scene " + std::to_string(k) + ": " + m;
        st = APBF_ERR_INVALID_ARG;
        if (k == 0) {
            sc = sk;
        } else {
            if (!same_physics(descs[0], descs[k]))
                return "scene " + std::to_string(k) + " differs from scene 0 in a physics parameter";
        }
        if (count > 1 && sk.fx_e != fx_exponent_for_h(descs[k].h)) {
            // a batch shares one fixed-point unit, the one a scene of that h takes alone
            st = APBF_ERR_NOT_SUPPORTED;
            return "scene " + std::to_string(k) + ": its grid spans 8e8 or more fixed-point units of 2^" +
                   std::to_string(fx_exponent_for_h(descs[k].h)) + " m on an axis; such scenes step alone, "
                   "not in a batch";
        }
        SceneGeom &g = geo[k];
        for (int ax = 0; ax < 3; ++ax)
            g.glo[ax] = sk.glo[ax];
        g.nx = sk.nx;
        g.ny = sk.ny;
        g.nz = sk.nz;
        g.cell_base = (uint32_t)c_total;
        g.p0 = (uint32_t)n_total;
        g.n = sk.n;
        n_total += sk.n;
        c_total += sk.ncell;
    }
    if (n_total >= kMaxParticles)
        return "the batch holds 2^31 - 1 particles or more";
    if (c_total >= (1ull << 31))
        return "the batch's grids hold too many cells";
    sc.n = (uint32_t)n_total;
    sc.ncell = (uint32_t)c_total;
    sc.scenes = count;
    sc.level_tiles = level_tile_count(sc.n);
    st = APBF_OK;
    return "";
}

struct Layout {
    size_t total = 0;
    size_t off[40] = {};
    int k = 0;
    size_t add(size_t bytes)
    {
        size_t o = total;
        total = align_up(total + (bytes ? bytes : 1));
        off[k++] = o;
        return o;
    }
};

}  // namespace

namespace apbf {
// The texture object over xt (raw 32-bit words, no conversion): the velocity
// pass gathers each neighbour's record of recA with plain loads and of xt
// through the texture path (measured on the 1M-particle ocean: 116.7 -> 100.3
// us per step; the same split in the solver passes, which gather one record
// per pair, was slower). An xt longer than the device's linear texture width
// gets none, and the pass then reads it with plain loads.
cudaError_t make_xt_texture(const StepConst &sc, Buffers &b)
{
    int dev = 0, maxw = 0, align = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture1DLinearWidth, dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&align, cudaDevAttrTextureAlignment, dev);
    if (e != cudaSuccess)
        return e;
    const size_t recs = (size_t)(sc.n ? sc.n : 1) + 1;
    const uintptr_t p = (uintptr_t)b.xt, base = align > 0 ? p / (uintptr_t)align * (uintptr_t)align : p;
    const size_t off = (p - base) / 16;
    if (align <= 0 || (p - base) % 16 || off + recs > (size_t)maxw)
        return cudaSuccess;  // no texture: the velocity pass reads xt with plain loads
    cudaResourceDesc rd = {};
    rd.resType = cudaResourceTypeLinear;
    rd.res.linear.devPtr = (void *)base;
    rd.res.linear.desc = cudaCreateChannelDesc<uint4>();
    rd.res.linear.sizeInBytes = 16 * (off + recs);
    cudaTextureDesc td = {};
    td.readMode = cudaReadModeElementType;
    if ((e = cudaCreateTextureObject(&b.texXt.t, &rd, &td, nullptr)) != cudaSuccess)
        return e;
    b.texXt.off = (uint32_t)off;
    return cudaSuccess;
}

// Carves the arena; with base == nullptr only measures.
size_t carve(const StepConst &sc, char *base, Buffers &b)
{
    const size_t n = sc.n ? sc.n : 1;
    const size_t ncell4 = (sc.ncell + 3) / 4 * 4;
    const size_t tiles = (sc.ncell + kScanTile - 1) / kScanTile;
    const size_t lvl_e = (size_t)sc.K * (sc.level_tiles ? sc.level_tiles : 1);
    const size_t dblocks = (n + kBlock - 1) / kBlock;
    Layout L;
    auto P = [&](size_t bytes) -> char * { size_t o = L.add(bytes); return base ? base + o : nullptr; };
    b.state_x = (float4 *)P(16 * n);
    b.state_v = (float4 *)P(16 * n);
    b.state_id = (uint32_t *)P(4 * n);
    b.key = (uint32_t *)P(4 * n);
    b.slot = (uint32_t *)P(4 * n);
    b.lvl = (uint8_t *)P(n);
    b.cnt = (uint32_t *)P(4 * ncell4);
    b.start = (uint32_t *)P(4 * (size_t)(sc.ncell + 1));
    b.tile_sums = (uint32_t *)P(4 * tiles);
    b.tmp = (uint32_t *)P(4 * n);
    b.recA = (float4 *)P(16 * (n + 1));
    b.recB = (float4 *)P(16 * (n + 1));
    b.xs32 = (float4 *)P(16 * (n + kEntryBlock));  // slack: the neighbour search reads whole batches
    b.xt = (float4 *)P(16 * (n + 1));
    b.id_s = (uint32_t *)P(4 * n);
    b.cell_s = (uint32_t *)P(4 * n);
    b.lvl_s = (uint8_t *)P(n);
    b.nbr_cnt = (uint8_t *)P(n);
    b.prev_cnt = (uint8_t *)P(n);
    b.nbr = (uint32_t *)P(4 * (size_t)list_rows(sc.max_nbr) * n);
    b.rho = (float *)P(4 * n);
    b.lodd = (float *)P(4 * n);
    b.act = (uint32_t *)P(4 * n);
    b.lvl_off = (uint32_t *)P(4 * lvl_e);
    b.lvl_count = (uint32_t *)P(4 * 258);
    // zeroed together at the start of every step (step_zero_bytes): the level
    // counts per tile, the distance range and the step's pair counters
    b.lvl_hist = (uint32_t *)P(4 * lvl_e);
    b.drange = (uint32_t *)P(8 * (size_t)sc.scenes);
    b.counters = (unsigned long long *)P(8 * kCounterSlots);
    b.err = (uint32_t *)P(4);
    b.err_scene = (uint32_t *)P(4 * (size_t)sc.scenes);
    b.dbg = (uint32_t *)P(16);
    b.dyn = (DynParams *)P(sizeof(DynParams) * (size_t)sc.scenes);
    b.geo = (const SceneGeom *)P(sizeof(SceneGeom) * (size_t)sc.scenes);
    b.sid = (const uint16_t *)P(2 * n);
    b.snap_x = (float4 *)P(16 * n);
    b.snap_v = (float4 *)P(16 * n);
    b.snap_id = (uint32_t *)P(4 * n);
    b.stage_f = (float *)P(12 * n);
    b.stage_u8 = (uint8_t *)P(n);
    b.dbg4 = (float4 *)P(16 * n);
    b.partials = (double *)P(32 * dblocks);
    b.dstats = (double *)P(32);
    return L.total;
}
}  // namespace apbf

namespace {

cudaEvent_t get_event(apbf_scene *s)
{
    if (!s->ev_pool.empty()) {
        cudaEvent_t e = s->ev_pool.back();
        s->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Runs one launch group, bracketed by timing events when timing is on.
template <typename F>
cudaError_t timed(apbf_scene *s, cudaStream_t st, uint32_t stage, F &&fn)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (s->timing) {
        a = get_event(s);
        b = get_event(s);
        cudaEventRecord(a, st);
    }
    cudaError_t e = fn();
    if (s->timing) {
        cudaEventRecord(b, st);
        s->timed.push_back({stage, a, b});
    }
    return e;
}

constexpr uint32_t kStageAll = 0xffffffffu;

// Enqueue one step of Fig. 7 on `st`, stopping after `stop_stage` (at
// iteration `stop_iter` for the lambda / delta-p stages).
apbf_status enqueue_step(apbf_scene *s, cudaStream_t st, uint32_t stop_stage, uint32_t stop_iter)
{
    const StepConst &sc = s->sc;
    const Buffers &b = s->b;
    const bool dtvs = sc.lod_mode == APBF_LOD_DTVS;
    cudaError_t e;
    if (dtvs && (!s->view_set || !s->view.depth || !s->view.ray))
        return fail(s, APBF_ERR_BAD_STATE, "a DTVS scene needs apbf_set_view before it steps");
    // one fill resets the level counts per tile, the distance range and the pair counters
    if ((e = cudaMemsetAsync(b.lvl_hist, 0, step_zero_bytes(b), st)) != cudaSuccess)
        return cuda_fail(s, e, "step counters");
    if (dtvs) {  // depth image, distances behind the visible surface and their range
        e = timed(s, st, APBF_STAGE_LOD_RANGE, [&] { return launch_dtvs(sc, b, s->view, s->sms, st); });
        if (e != cudaSuccess)
            return cuda_fail(s, e, "dtvs");
    }
    if (stop_stage == APBF_STAGE_LOD_RANGE)
        return APBF_OK;
    if ((e = timed(s, st, APBF_STAGE_PREDICT, [&] { return launch_predict_hash(sc, b, st, false); })) != cudaSuccess)
        return cuda_fail(s, e, "predict_hash");
    if (stop_stage == APBF_STAGE_PREDICT)
        return APBF_OK;
    if ((e = timed(s, st, APBF_STAGE_SCAN, [&] { return launch_scan(sc, b, st); })) != cudaSuccess)
        return cuda_fail(s, e, "scan");
    if (stop_stage == APBF_STAGE_SCAN)
        return APBF_OK;
    if ((e = timed(s, st, APBF_STAGE_SCATTER, [&] { return launch_scatter(sc, b, st); })) != cudaSuccess)
        return cuda_fail(s, e, "scatter");
    if (stop_stage == APBF_STAGE_SCATTER)
        return APBF_OK;
    if ((e = timed(s, st, APBF_STAGE_REORDER, [&] { return launch_reorder(sc, b, st, false); })) != cudaSuccess)
        return cuda_fail(s, e, "reorder");
    s->cur_buf = 0;
    if (stop_stage == APBF_STAGE_REORDER)
        return APBF_OK;
    // the level partition comes first: the neighbour lists are stored by active-list position
    const bool part = partitioned(sc);
    if (part) {
        if ((e = timed(s, st, APBF_STAGE_LEVELS, [&] { return launch_levels(sc, b, st); })) != cudaSuccess)
            return cuda_fail(s, e, "levels");
    }
    if (stop_stage == APBF_STAGE_LEVELS)
        return APBF_OK;
    e = timed(s, st, APBF_STAGE_NEIGHBORS, [&] { return launch_neighbors(sc, b, st, part); });
    s->lists_by_slot = !part;
    if (e != cudaSuccess)
        return cuda_fail(s, e, "neighbors");
    if (stop_stage == APBF_STAGE_NEIGHBORS)
        return APBF_OK;
    if (sc.stabil_s > 1 && sc.stabil_iters > 0) {
        if ((e = timed(s, st, APBF_STAGE_PRESTAB, [&] { return launch_prestab(sc, b, st); })) != cudaSuccess)
            return cuda_fail(s, e, "prestab");
    }
    if (stop_stage == APBF_STAGE_PRESTAB)
        return APBF_OK;
    for (uint32_t l = 1; l <= sc.n_max; ++l) {
        const bool dense = l <= sc.n_min;
        e = timed(s, st, APBF_STAGE_LAMBDA, [&] { return launch_lambda(sc, b, st, l, dense, s->grid_iter, s->tune); });
        if (e != cudaSuccess)
            return cuda_fail(s, e, "lambda");
        s->cur_buf = 1;
        if (stop_stage == APBF_STAGE_LAMBDA && stop_iter == l)
            return APBF_OK;
        e = timed(s, st, APBF_STAGE_DELTAP, [&] { return launch_deltap(sc, b, st, l, dense, s->grid_iter, s->tune); });
        if (e != cudaSuccess)
            return cuda_fail(s, e, "deltap");
        s->cur_buf = 0;
        if (stop_stage == APBF_STAGE_DELTAP && stop_iter == l)
            return APBF_OK;
    }
    if ((e = timed(s, st, APBF_STAGE_FINALIZE, [&] { return launch_finalize(sc, b, st); })) != cudaSuccess)
        return cuda_fail(s, e, "finalize");
    return APBF_OK;
}

apbf_status upload_dyn(apbf_scene *s)
{
    if (!s->dyn_dirty)
        return APBF_OK;
    int k = s->dyn_slot;
    s->dyn_slot = (s->dyn_slot + 1) % 16;
    APBF_CUDA(s, cudaEventSynchronize(s->dyn_ev[k]));  // the previous copy out of this slot is done
    const size_t cnt = s->dyn.size();  // <= dyn_cap, the stride of the ring's slots
    std::memcpy(s->dyn_pinned + k * s->dyn_cap, s->dyn.data(), sizeof(DynParams) * cnt);
    APBF_CUDA(s, cudaMemcpyAsync(s->b.dyn, s->dyn_pinned + k * s->dyn_cap, sizeof(DynParams) * cnt,
                                 cudaMemcpyHostToDevice, s->stream));
    APBF_CUDA(s, cudaEventRecord(s->dyn_ev[k], s->stream));
    s->dyn_dirty = false;
    return APBF_OK;
}

apbf_status check_device_errors(apbf_scene *s)
{
    uint32_t *h = (uint32_t *)s->pinned_small;
    APBF_CUDA(s, cudaMemcpyAsync(h, s->b.err, 4, cudaMemcpyDeviceToHost, s->stream));
    APBF_CUDA(s, cudaStreamSynchronize(s->stream));
    if (*h & kErrDebugCheck) {
        static const char *what[] = {"?", "cell key outside the grid", "cell counts do not add up to n",
                                     "sorted slot outside its cell's range", "active count above n or not nested",
                                     "neighbour entry beyond the padding record"};
        uint32_t dbg[2] = {0, 0};
        APBF_CUDA(s, cudaMemcpy(dbg, s->b.dbg, 8, cudaMemcpyDeviceToHost));
        return fail(s, APBF_ERR_CHECK_FAILED, std::string("debug check ") + std::to_string(dbg[0]) + " (" +
                                                  what[dbg[0] < 6 ? dbg[0] : 0] + ") failed at index " +
                                                  std::to_string(dbg[1]));
    }
    if (*h & kErrNeighborOverflow)
        return fail(s, APBF_ERR_NEIGHBOR_OVERFLOW,
                    "a particle had more neighbours than max_neighbors (" + std::to_string(s->sc.max_nbr) + ")");
    return APBF_OK;
}

apbf_status enter(apbf_scene *s)
{
    if (!s)
        return APBF_ERR_INVALID_ARG;
    if (s->sticky != APBF_OK)
        return s->sticky;
    int dev = -1;
    if (cudaGetDevice(&dev) == cudaSuccess && dev != s->device)
        APBF_CUDA(s, cudaSetDevice(s->device));
    return APBF_OK;
}

apbf_status build_graph(apbf_scene *s)
{
    APBF_CUDA(s, cudaStreamBeginCapture(s->capture_stream, cudaStreamCaptureModeThreadLocal));
    apbf_status st = enqueue_step(s, s->capture_stream, kStageAll, 0);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->capture_stream, &g);
    if (st != APBF_OK) {
        if (g)
            cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess)
        return cuda_fail(s, e, "cudaStreamEndCapture");
    s->graph = g;
    APBF_CUDA(s, cudaGraphInstantiate(&s->gexec, g, 0));
    return APBF_OK;
}

}  // namespace

namespace apbf {
// Message returned by apbf_last_error(NULL) for calls that have no scene.
void set_last_error_message(const std::string &m) { g_create_error = m; }
}  // namespace apbf

extern "C" {

APBF_API const char *apbf_status_string(apbf_status st)
{
    switch (st) {
    case APBF_OK: return "ok";
    case APBF_ERR_INVALID_ARG: return "invalid argument";
    case APBF_ERR_OUT_OF_MEMORY: return "out of device memory";
    case APBF_ERR_CUDA: return "CUDA error";
    case APBF_ERR_TIMEOUT: return "device wait timed out";
    case APBF_ERR_BAD_STATE: return "bad state";
    case APBF_ERR_NEIGHBOR_OVERFLOW: return "neighbour list overflow";
    case APBF_ERR_NOT_SUPPORTED: return "not supported";
    case APBF_ERR_CHECK_FAILED: return "debug check failed";
    }
    return "unknown status";
}

APBF_API apbf_status apbf_rest_density(float h, float mass, float spacing, double *rho0)
{
    if (!rho0 || !(h > 0.0f) || !(mass > 0.0f) || !(spacing > 0.0f) || !std::isfinite(h) || !std::isfinite(spacing))
        return APBF_ERR_INVALID_ARG;
    // Eq. 6 summed over the lattice points within h of the centre particle.
    const double PI = 3.14159265358979323846;
    const double hd = h, s = spacing, c = 315.0 / (64.0 * PI * std::pow(hd, 9));
    const int r = (int)std::ceil(hd / s) + 1;
    double sum = 0.0;
    for (int i = -r; i <= r; ++i)
        for (int j = -r; j <= r; ++j)
            for (int k = -r; k <= r; ++k) {
                double d2 = (double)(i * i + j * j + k * k) * s * s;
                double u = hd * hd - d2;
                if (u > 0.0)
                    sum += u * u * u;
            }
    *rho0 = (double)mass * c * sum;
    return APBF_OK;
}

APBF_API apbf_status apbf_batch_bytes(const apbf_scene_desc *descs, uint32_t count, size_t *bytes)
{
    if (!bytes)
        return fail(nullptr, APBF_ERR_INVALID_ARG, "bytes is NULL");
    StepConst sc;
    std::vector<SceneGeom> geo;
    apbf_status st;
    std::string m = derive_batch(descs, count, sc, geo, st);
    if (st != APBF_OK)
        return fail(nullptr, st, m);
    Buffers b;
    *bytes = carve(sc, nullptr, b);
    return APBF_OK;
}

APBF_API apbf_status apbf_scene_bytes(const apbf_scene_desc *desc, size_t *bytes)
{
    return apbf_batch_bytes(desc, 1, bytes);
}

}  // extern "C"

namespace apbf {
// A scene object whose arena is carved for `cap` (particles, cells, scenes of
// the largest membership it will hold), zeroed on its stream; nothing is
// uploaded and no geometry is set.
apbf_status alloc_scene(const StepConst &cap, uint32_t flags, void *cuda_stream, void *device_arena,
                        size_t arena_bytes, apbf_scene **out, std::string &msg)
{
    *out = nullptr;
    if (device_arena && ((uintptr_t)device_arena % kAlign)) {
        msg = "device_arena must be 256-byte aligned";
        return APBF_ERR_INVALID_ARG;
    }
    apbf_scene *s = new (std::nothrow) apbf_scene();
    if (!s) {
        msg = "host allocation failed";
        return APBF_ERR_OUT_OF_MEMORY;
    }
    s->sc = cap;
    s->dyn_cap = cap.scenes;
    s->flags = flags;
    s->stream = (cudaStream_t)cuda_stream;
    auto bail = [&](apbf_status code, const std::string &m) {
        msg = m;
        apbf_destroy_scene(s);
        return code;
    };
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess)
        return bail(APBF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    const size_t need = carve(cap, nullptr, s->b);
    if (device_arena) {
        if (arena_bytes < need)
            return bail(APBF_ERR_OUT_OF_MEMORY, "device_arena is smaller than the bytes the scene needs");
        s->arena = device_arena;
        s->arena_bytes = arena_bytes;
    } else {
        e = cudaMalloc(&s->arena, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->arena = nullptr;
            return bail(APBF_ERR_OUT_OF_MEMORY, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        s->own_arena = true;
        s->arena_bytes = need;
    }
    carve(cap, (char *)s->arena, s->b);
    if ((e = make_xt_texture(cap, s->b)) != cudaSuccess)
        return bail(APBF_ERR_CUDA, std::string("cudaCreateTextureObject: ") + cudaGetErrorString(e));
    if ((e = cudaHostAlloc(&s->pinned_small, 4096, cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaHostAlloc((void **)&s->dyn_pinned, 16 * sizeof(DynParams) * (size_t)cap.scenes,
                           cudaHostAllocDefault)) != cudaSuccess)
        return bail(APBF_ERR_CUDA, std::string("cudaHostAlloc: ") + cudaGetErrorString(e));
    for (int k = 0; k < 16; ++k)
        if ((e = cudaEventCreateWithFlags(&s->dyn_ev[k], cudaEventDisableTiming)) != cudaSuccess)
            return bail(APBF_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
    if ((e = cudaStreamCreateWithFlags(&s->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(APBF_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    if ((e = cudaMemsetAsync(s->arena, 0, need, s->stream)) != cudaSuccess)
        return bail(APBF_ERR_CUDA, std::string("arena memset: ") + cudaGetErrorString(e));
    s->grid_iter = s->sms > 0 ? s->sms : 1;  // the launchers scale by each kernel's occupancy
    *out = s;
    return APBF_OK;
}
}  // namespace apbf

extern "C" {

APBF_API apbf_status apbf_create_batch(const apbf_scene_desc *descs, uint32_t count, void *cuda_stream,
                                       void *device_arena, size_t arena_bytes, apbf_scene **out)
{
    if (!out)
        return fail(nullptr, APBF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    StepConst sc;
    std::vector<SceneGeom> geo;
    apbf_status st;
    std::string m = derive_batch(descs, count, sc, geo, st);
    if (st != APBF_OK)
        return fail(nullptr, st, m);
    for (uint32_t k = 0; k < count; ++k) {
        const apbf_scene_desc *d = descs + k;
        const std::string who = count > 1 ? "scene " + std::to_string(k) + ": " : "";
        for (uint32_t i = 0; i < 3 * d->n; ++i)
            if (!std::isfinite(d->pos[i]) || (d->vel && !std::isfinite(d->vel[i])))
                return fail(nullptr, APBF_ERR_INVALID_ARG, who + "positions and velocities must be finite");
        for (uint32_t i = 0; i < d->n; ++i)
            for (int a = 0; a < 3; ++a)
                if (!(d->pos[3 * i + a] >= d->grid_lo[a] && d->pos[3 * i + a] <= d->grid_hi[a]))
                    return fail(nullptr, APBF_ERR_INVALID_ARG,
                                who + "particle " + std::to_string(i) + " lies outside the grid");
    }
    apbf_scene *s = nullptr;
    std::string amsg;
    st = alloc_scene(sc, descs[0].flags, cuda_stream, device_arena, arena_bytes, &s, amsg);
    if (st != APBF_OK)
        return fail(nullptr, st, amsg);
    s->geo = geo;
    s->grid_hi3.resize(3 * (size_t)count);
    s->dyn.assign(count, DynParams{});
    for (uint32_t k = 0; k < count; ++k)
        for (int a = 0; a < 3; ++a) {
            s->grid_hi3[3 * k + a] = descs[k].grid_hi[a];
            s->dyn[k].box_lo[a] = descs[k].box_lo[a];
            s->dyn[k].box_hi[a] = descs[k].box_hi[a];
            s->dyn[k].dir[a] = a == 0 ? 1.0f : 0.0f;
            s->dyn[k].auto_range = 1;
        }
    auto bail = [&](apbf_status code, const std::string &msg) {
        g_create_error = msg;
        apbf_destroy_scene(s);
        return code;
    };
    cudaError_t e;
    const Buffers &b = s->b;
    const size_t n = sc.n;

    // initial state: the scenes' particles concatenated, each in its id order;
    // global id = scene's first slot + id within the scene
    std::vector<float4> hx(n ? n : 1), hv(n ? n : 1);
    std::vector<uint32_t> hid(n ? n : 1);
    std::vector<uint16_t> hsid(n ? n : 1);
    for (uint32_t k = 0; k < count; ++k) {
        const apbf_scene_desc *d = descs + k;
        for (size_t i = 0; i < d->n; ++i) {
            const size_t g = geo[k].p0 + i;
            hx[g] = make_float4(d->pos[3 * i], d->pos[3 * i + 1], d->pos[3 * i + 2], 0.0f);
            hv[g] = d->vel ? make_float4(d->vel[3 * i], d->vel[3 * i + 1], d->vel[3 * i + 2], 0.0f)
                           : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            hid[g] = (uint32_t)g;
            hsid[g] = (uint16_t)k;
        }
    }
    std::vector<uint32_t> lc(258, 0u);
    for (uint32_t l = 0; l <= sc.n_max; ++l)
        lc[l] = sc.n;  // every particle is active in every iteration until a partition says otherwise
    cudaStream_t st0 = s->stream;
    if ((e = cudaMemcpyAsync(b.state_x, hx.data(), 16 * n, cudaMemcpyHostToDevice, st0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b.state_v, hv.data(), 16 * n, cudaMemcpyHostToDevice, st0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b.state_id, hid.data(), 4 * n, cudaMemcpyHostToDevice, st0)) != cudaSuccess ||
        (e = cudaMemcpyAsync((void *)b.sid, hsid.data(), 2 * n, cudaMemcpyHostToDevice, st0)) != cudaSuccess ||
        (e = cudaMemcpyAsync((void *)b.geo, geo.data(), sizeof(SceneGeom) * count, cudaMemcpyHostToDevice, st0)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(b.lvl_count, lc.data(), 4 * 258, cudaMemcpyHostToDevice, st0)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st0)) != cudaSuccess)
        return bail(APBF_ERR_CUDA, std::string("initial upload: ") + cudaGetErrorString(e));
    s->dyn_dirty = true;
    *out = s;
    return APBF_OK;
}

APBF_API apbf_status apbf_create_scene(const apbf_scene_desc *d, void *cuda_stream, void *device_arena,
                                       size_t arena_bytes, apbf_scene **out)
{
    return apbf_create_batch(d, 1, cuda_stream, device_arena, arena_bytes, out);
}

namespace {
// The DTVS camera basis needs dir != 0 and dir x up != 0 (checked in FP64).
bool view_axes_ok(const float dir[3], const float *up)
{
    const double d0 = dir[0], d1 = dir[1], d2 = dir[2];
    if (d0 * d0 + d1 * d1 + d2 * d2 == 0.0)
        return false;
    if (!up)
        return true;
    const double c0 = d1 * up[2] - d2 * up[1], c1 = d2 * up[0] - d0 * up[2], c2 = d0 * up[1] - d1 * up[0];
    return c0 * c0 + c1 * c1 + c2 * c2 > 1e-24 * (d0 * d0 + d1 * d1 + d2 * d2);
}

apbf_status set_camera_range(apbf_scene *s, uint32_t k0, uint32_t k1, const float eye[3], const float dir[3],
                             float d_near, float d_far)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (!eye || !dir || !finite3(eye) || !finite3(dir) || !std::isfinite(d_near) || !std::isfinite(d_far))
        return fail(s, APBF_ERR_INVALID_ARG, "camera values must be finite and non-NULL");
    if (k0 >= s->sc.scenes)
        return fail(s, APBF_ERR_INVALID_ARG, "scene index out of range");
    if (s->sc.lod_mode == APBF_LOD_DTVS && !view_axes_ok(dir, s->view_set ? s->view.up : nullptr))
        return fail(s, APBF_ERR_INVALID_ARG, "dir must be non-zero and not parallel to the view's up vector");
    for (uint32_t k = k0; k < k1; ++k) {
        for (int a = 0; a < 3; ++a) {
            s->dyn[k].eye[a] = eye[a];
            s->dyn[k].dir[a] = dir[a];
        }
        s->dyn[k].d_near = d_near;
        s->dyn[k].d_far = d_far;
        s->dyn[k].auto_range = (d_near < d_far) ? 0u : 1u;
    }
    s->dyn_dirty = true;
    return APBF_OK;
}

apbf_status set_box_range(apbf_scene *s, uint32_t k0, uint32_t k1, const float lo[3], const float hi[3])
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (!lo || !hi || !finite3(lo) || !finite3(hi))
        return fail(s, APBF_ERR_INVALID_ARG, "box bounds must be finite and non-NULL");
    if (k0 >= s->sc.scenes)
        return fail(s, APBF_ERR_INVALID_ARG, "scene index out of range");
    for (uint32_t k = k0; k < k1; ++k)
        for (int a = 0; a < 3; ++a)
            if (!(s->geo[k].glo[a] <= lo[a] && lo[a] < hi[a] && hi[a] <= s->grid_hi3[3 * k + a]))
                return fail(s, APBF_ERR_INVALID_ARG, "need grid_lo <= lo < hi <= grid_hi on every axis");
    for (uint32_t k = k0; k < k1; ++k)
        for (int a = 0; a < 3; ++a) {
            s->dyn[k].box_lo[a] = lo[a];
            s->dyn[k].box_hi[a] = hi[a];
        }
    s->dyn_dirty = true;
    return APBF_OK;
}
}  // namespace

APBF_API apbf_status apbf_set_camera(apbf_scene *s, const float eye[3], const float dir[3], float d_near, float d_far)
{
    return s ? set_camera_range(s, 0, s->sc.scenes, eye, dir, d_near, d_far) : APBF_ERR_INVALID_ARG;
}

APBF_API apbf_status apbf_set_camera_at(apbf_scene *s, uint32_t index, const float eye[3], const float dir[3],
                                        float d_near, float d_far)
{
    return s ? set_camera_range(s, index, index + 1, eye, dir, d_near, d_far) : APBF_ERR_INVALID_ARG;
}

APBF_API apbf_status apbf_set_box(apbf_scene *s, const float lo[3], const float hi[3])
{
    return s ? set_box_range(s, 0, s->sc.scenes, lo, hi) : APBF_ERR_INVALID_ARG;
}

APBF_API apbf_status apbf_set_obstacles(apbf_scene *s, uint32_t index, const apbf_obstacle *obstacles,
                                        uint32_t count)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (index >= s->sc.scenes)
        return fail(s, APBF_ERR_INVALID_ARG, "scene index out of range");
    if (count > APBF_MAX_OBSTACLES || (count && !obstacles))
        return fail(s, APBF_ERR_INVALID_ARG, "need count <= APBF_MAX_OBSTACLES and a non-NULL array");
    for (uint32_t k = 0; k < count; ++k) {
        const apbf_obstacle &o = obstacles[k];
        if (!finite3(o.a) || !finite3(o.b))
            return fail(s, APBF_ERR_INVALID_ARG, "obstacle values must be finite");
        bool ok = false;
        if (o.kind == APBF_OBSTACLE_SPHERE)
            ok = o.b[0] > 0.0f;
        else if (o.kind == APBF_OBSTACLE_BOX)
            ok = o.a[0] < o.b[0] && o.a[1] < o.b[1] && o.a[2] < o.b[2];
        else if (o.kind == APBF_OBSTACLE_CONE)
            ok = o.b[0] > 0.0f && o.b[1] > 0.0f;
        if (!ok)
            return fail(s, APBF_ERR_INVALID_ARG, "obstacle " + std::to_string(k) + ": unknown kind or bad size");
    }
    DynParams &d = s->dyn[index];
    d.n_obst = count;
    for (uint32_t k = 0; k < APBF_MAX_OBSTACLES; ++k) {
        Obstacle o{};
        if (k < count) {
            o.kind = obstacles[k].kind;
            for (int a = 0; a < 3; ++a) {
                o.a[a] = obstacles[k].a[a];
                o.b[a] = obstacles[k].b[a];
            }
        }
        d.obst[k] = o;
    }
    s->dyn_dirty = true;
    return APBF_OK;
}

APBF_API apbf_status apbf_set_box_at(apbf_scene *s, uint32_t index, const float lo[3], const float hi[3])
{
    return s ? set_box_range(s, index, index + 1, lo, hi) : APBF_ERR_INVALID_ARG;
}

APBF_API apbf_status apbf_set_view(apbf_scene *s, uint32_t width, uint32_t height, float tan_half_fov,
                                   const float up[3], float radius)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (s->sc.lod_mode != APBF_LOD_DTVS)
        return fail(s, APBF_ERR_INVALID_ARG, "the scene's lod_mode is not APBF_LOD_DTVS");
    if (width < 1 || height < 1 || width > 16384 || height > 16384 || (uint64_t)width * height > (1ull << 26))
        return fail(s, APBF_ERR_INVALID_ARG, "need 1 <= width, height <= 16384 and width*height <= 2^26");
    if (!(tan_half_fov > 0.0f) || !(tan_half_fov < 1.0e4f) || !(radius > 0.0f) || !std::isfinite(radius))
        return fail(s, APBF_ERR_INVALID_ARG, "need 0 < tan_half_fov < 1e4 and a finite radius > 0");
    if (!up || !finite3(up) || !view_axes_ok(s->dyn[0].dir, up))
        return fail(s, APBF_ERR_INVALID_ARG, "up must be finite and not parallel to the camera direction");
    APBF_CUDA(s, cudaStreamSynchronize(s->stream));  // the previous image may still be in use
    // one allocation: depth, rays, tile counters, starts and lists, the big-sphere list
    const size_t pix = (size_t)width * height;
    const uint32_t tx = (width + kTilePx - 1) / kTilePx, ty = (height + kTilePx - 1) / kTilePx;
    const size_t tiles = (size_t)tx * ty, n = s->sc.n;
    const size_t cap = (size_t)kSplatListPerParticle * n + 65536;
    size_t off[16], total = 0;
    const size_t sizes[16] = {4 * pix, 16 * pix, 4 * tiles, 4 * tiles, 4 * (tiles + 1), 4 * cap, 4 * n, 4,
                              4 * (tiles + 1), 8, n, 8 * n, 4 * n, 4 * tiles, 4 * n,
                              4 * (tiles + cap / kSplatChunk + 1)};
    for (int k = 0; k < 16; ++k) {
        off[k] = total;
        total = align_up(total + (sizes[k] ? sizes[k] : 1));
    }
    if (!s->view.alloc || s->view.alloc_bytes < total) {
        if (s->view.alloc)
            cudaFree(s->view.alloc);
        s->view.alloc = nullptr;
        s->view.alloc_bytes = 0;
        s->view_set = false;
        cudaError_t e = cudaMalloc(&s->view.alloc, total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->view.alloc = nullptr;
            return fail(s, APBF_ERR_OUT_OF_MEMORY, std::string("view image: ") + cudaGetErrorString(e));
        }
        s->view.alloc_bytes = total;
    }
    char *base = (char *)s->view.alloc;
    s->view.depth = (uint32_t *)(base + off[0]);
    s->view.ray = (float4 *)(base + off[1]);
    s->view.tile_cnt = (uint32_t *)(base + off[2]);
    s->view.tile_fill = (uint32_t *)(base + off[3]);
    s->view.tile_start = (uint32_t *)(base + off[4]);
    s->view.tile_list = (uint32_t *)(base + off[5]);
    s->view.big = (uint32_t *)(base + off[6]);
    s->view.big_cnt = (uint32_t *)(base + off[7]);
    s->view.chunk_start = (uint32_t *)(base + off[8]);
    s->view.list_used = (unsigned long long *)(base + off[9]);
    s->view.accepted = (uint8_t *)(base + off[10]);
    s->view.box = (uint2 *)(base + off[11]);
    s->view.near = (float *)(base + off[12]);
    s->view.tile_max = (uint32_t *)(base + off[13]);
    s->view.open_mask = (uint32_t *)(base + off[14]);
    s->view.chunk_tile = (uint32_t *)(base + off[15]);
    s->view.list_cap = (uint32_t)cap;
    s->view.tiles_x = tx;
    s->view.tiles_y = ty;
    s->view.W = width;
    s->view.H = height;
    s->view.tan_half = tan_half_fov;
    for (int a = 0; a < 3; ++a)
        s->view.up[a] = up[a];
    s->view.radius = radius;
    {
        const double ax = (double)tan_half_fov * width / height, ay = tan_half_fov;
        const double g = std::atan(std::sqrt(ax * ax + ay * ay)) + 0.01;
        // the cosine form of the cull holds while gamma + beta <= pi (beta <= pi/2)
        s->view.cull_cos = g < 1.5 ? (float)std::cos(g) : -1.0e30f;
        s->view.cull_sin = g < 1.5 ? (float)std::sin(g) : 0.0f;
    }
    s->view_set = true;
    drop_graph(s);
    return APBF_OK;
}

APBF_API apbf_status apbf_set_view_outside_level(apbf_scene *s, uint32_t level)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (s->sc.lod_mode != APBF_LOD_DTVS)
        return fail(s, APBF_ERR_INVALID_ARG, "the scene's lod_mode is not APBF_LOD_DTVS");
    if (level == 0)
        level = s->sc.n_min;
    if (level < s->sc.n_min || level > s->sc.n_max)
        return fail(s, APBF_ERR_INVALID_ARG, "need level = 0 or n_min <= level <= n_max");
    if (level != s->sc.dtvs_outside) {
        s->sc.dtvs_outside = level;
        drop_graph(s);  // the captured step holds the step constants
    }
    return APBF_OK;
}

APBF_API apbf_status apbf_step(apbf_scene *s, uint32_t nsteps)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (s->sc.n == 0) {
        s->stepped = true;
        return APBF_OK;
    }
    if (s->sc.lod_mode == APBF_LOD_DTVS && !s->view_set)
        return fail(s, APBF_ERR_BAD_STATE, "a DTVS scene needs apbf_set_view before it steps");
    const bool eager = s->timing || (s->flags & APBF_FLAG_NO_GRAPH);
    for (uint32_t k = 0; k < nsteps; ++k) {
        if ((st = upload_dyn(s)) != APBF_OK)
            return st;
        if (eager) {
            if ((st = enqueue_step(s, s->stream, kStageAll, 0)) != APBF_OK)
                return st;
        } else {
            if (!s->gexec && (st = build_graph(s)) != APBF_OK)
                return st;
            APBF_CUDA(s, cudaGraphLaunch(s->gexec, s->stream));
        }
    }
    APBF_CUDA(s, cudaGetLastError());
    s->stepped = true;
    return APBF_OK;
}

APBF_API apbf_status apbf_read_state(apbf_scene *s, float *pos, float *vel, uint8_t *n_iter, float *rho)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if ((st = check_device_errors(s)) != APBF_OK)
        return st;
    const size_t n = s->sc.n;
    if (n == 0)
        return APBF_OK;
    if (s->copy_pending)  // the staging buffer may still be on its way to the host
        APBF_CUDA(s, cudaStreamWaitEvent(s->stream, s->copy_ev, 0));
    float *outs_f[3] = {pos, vel, nullptr};
    for (uint32_t what = 0; what < 2; ++what) {
        if (!outs_f[what])
            continue;
        APBF_CUDA(s, launch_unpermute(s->sc, s->b, s->stream, what));
        APBF_CUDA(s, cudaMemcpyAsync(outs_f[what], s->b.stage_f, 12 * n, cudaMemcpyDeviceToHost, s->stream));
    }
    if (n_iter) {
        APBF_CUDA(s, launch_unpermute(s->sc, s->b, s->stream, 2));
        APBF_CUDA(s, cudaMemcpyAsync(n_iter, s->b.stage_u8, n, cudaMemcpyDeviceToHost, s->stream));
    }
    if (rho) {
        APBF_CUDA(s, launch_unpermute(s->sc, s->b, s->stream, 3));
        APBF_CUDA(s, cudaMemcpyAsync(rho, s->b.stage_f, 4 * n, cudaMemcpyDeviceToHost, s->stream));
    }
    APBF_CUDA(s, cudaStreamSynchronize(s->stream));
    return APBF_OK;
}

APBF_API apbf_status apbf_read_positions_async(apbf_scene *s, float *pos)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (!pos)
        return fail(s, APBF_ERR_INVALID_ARG, "pos is NULL");
    const size_t n = s->sc.n;
    if (n == 0)
        return APBF_OK;
    if (!s->copy_stream) {
        APBF_CUDA(s, cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking));
        APBF_CUDA(s, cudaEventCreateWithFlags(&s->unperm_ev, cudaEventDisableTiming));
        APBF_CUDA(s, cudaEventCreateWithFlags(&s->copy_ev, cudaEventDisableTiming));
    }
    if (s->copy_pending)  // the previous copy still reads the staging buffer
        APBF_CUDA(s, cudaStreamWaitEvent(s->stream, s->copy_ev, 0));
    APBF_CUDA(s, launch_unpermute(s->sc, s->b, s->stream, 0));
    APBF_CUDA(s, cudaEventRecord(s->unperm_ev, s->stream));
    APBF_CUDA(s, cudaStreamWaitEvent(s->copy_stream, s->unperm_ev, 0));
    APBF_CUDA(s, cudaMemcpyAsync(pos, s->b.stage_f, 12 * n, cudaMemcpyDeviceToHost, s->copy_stream));
    APBF_CUDA(s, cudaEventRecord(s->copy_ev, s->copy_stream));
    s->copy_pending = true;
    return APBF_OK;
}

APBF_API apbf_status apbf_density_stats(apbf_scene *s, double stats[4])
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (!stats)
        return fail(s, APBF_ERR_INVALID_ARG, "stats is NULL");
    stats[0] = stats[1] = stats[2] = stats[3] = 0.0;
    if (s->sc.n == 0)
        return check_device_errors(s);
    Buffers bb = s->b;
    bb.counters = s->b.counters + kDiagCounterSlot;  // keep the step's counters
    cudaStream_t q = s->stream;
    int nb = 0;
    APBF_CUDA(s, launch_predict_hash(s->sc, bb, q, true));
    APBF_CUDA(s, launch_scan(s->sc, bb, q));
    APBF_CUDA(s, launch_scatter(s->sc, bb, q));
    APBF_CUDA(s, launch_reorder(s->sc, bb, q, true));
    APBF_CUDA(s, launch_neighbors(s->sc, bb, q, false));  // by sorted slot, for the density kernel
    s->lists_by_slot = true;
    APBF_CUDA(s, launch_density(s->sc, bb, q, &nb));
    double *h = (double *)s->pinned_small + 8;
    APBF_CUDA(s, cudaMemcpyAsync(h, s->b.dstats, 32, cudaMemcpyDeviceToHost, q));
    if ((st = check_device_errors(s)) != APBF_OK)
        return st;
    for (int k = 0; k < 4; ++k)
        stats[k] = h[k];
    return APBF_OK;
}

APBF_API apbf_status apbf_get_step_info(apbf_scene *s, apbf_step_info *info)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (!info)
        return fail(s, APBF_ERR_INVALID_ARG, "info is NULL");
    std::memset(info, 0, sizeof(*info));
    if ((st = check_device_errors(s)) != APBF_OK)
        return st;
    const StepConst &sc = s->sc;
    if (sc.n == 0 || !s->stepped)
        return APBF_OK;
    std::vector<unsigned long long> c(kCounterSlots);
    std::vector<uint32_t> lc(258);
    uint32_t dr[2];
    APBF_CUDA(s, cudaMemcpy(c.data(), s->b.counters, 8 * kCounterSlots, cudaMemcpyDeviceToHost));
    APBF_CUDA(s, cudaMemcpy(lc.data(), s->b.lvl_count, 4 * 258, cudaMemcpyDeviceToHost));
    APBF_CUDA(s, cudaMemcpy(&dr[0], s->b.drange, 4, cudaMemcpyDeviceToHost));
    APBF_CUDA(s, cudaMemcpy(&dr[1], s->b.drange + sc.scenes, 4, cudaMemcpyDeviceToHost));
    const bool partitioned = sc.lod_mode != APBF_LOD_FIXED && sc.K > 1;
    info->neighbor_pairs = c[0];  // without a partition; with one, the sum of the bins below
    info->total_particle_iterations = c[kIterTotalSlot];
    for (uint32_t l = 0; l < 256; ++l) {
        uint32_t a = 0;
        if (l <= sc.n_max)
            a = partitioned ? lc[l] : sc.n;
        info->active_count[l] = a;
        if (l >= 1)
            info->particle_iterations += a;
    }
    if (partitioned) {
        for (uint32_t bin = 0; bin < sc.K; ++bin) {
            info->neighbor_pairs += c[2 + bin];
            info->lambda_pairs += c[2 + bin] * (unsigned long long)(sc.n_max - bin);
        }
    } else {
        info->lambda_pairs = c[0] * (unsigned long long)sc.n_max;
    }
    if (sc.lod_mode != APBF_LOD_FIXED) {
        if (s->dyn[0].auto_range) {
            uint32_t lo = ~dr[0];  // the minimum is kept as the complement of its bit pattern
            std::memcpy(&info->d_range[0], &lo, 4);
            std::memcpy(&info->d_range[1], &dr[1], 4);
        } else {
            info->d_range[0] = s->dyn[0].d_near;
            info->d_range[1] = s->dyn[0].d_far;
        }
    }
    return APBF_OK;
}

APBF_API apbf_status apbf_sync(apbf_scene *s)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (s->copy_pending) {
        APBF_CUDA(s, cudaEventSynchronize(s->copy_ev));
        s->copy_pending = false;
    }
    return check_device_errors(s);
}

APBF_API const char *apbf_last_error(const apbf_scene *s)
{
    if (!s)
        return g_create_error.c_str();
    return s->msg.c_str();
}

APBF_API void apbf_destroy_scene(apbf_scene *s)
{
    if (!s)
        return;
    if (s->stream || s->arena)
        cudaStreamSynchronize(s->stream);
    if (s->copy_stream) {
        cudaStreamSynchronize(s->copy_stream);
        cudaStreamDestroy(s->copy_stream);
        cudaEventDestroy(s->unperm_ev);
        cudaEventDestroy(s->copy_ev);
    }
    if (s->gexec)
        cudaGraphExecDestroy(s->gexec);
    if (s->graph)
        cudaGraphDestroy(s->graph);
    if (s->capture_stream)
        cudaStreamDestroy(s->capture_stream);
    for (auto &t : s->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto e : s->ev_pool)
        cudaEventDestroy(e);
    for (int k = 0; k < 16; ++k)
        if (s->dyn_ev[k])
            cudaEventDestroy(s->dyn_ev[k]);
    if (s->dyn_pinned)
        cudaFreeHost(s->dyn_pinned);
    if (s->pinned_small)
        cudaFreeHost(s->pinned_small);
    if (s->b.texXt.t)
        cudaDestroyTextureObject(s->b.texXt.t);
    if (s->own_arena && s->arena)
        cudaFree(s->arena);
    if (s->view.alloc)
        cudaFree(s->view.alloc);
    delete s;
}

APBF_API apbf_status apbf_set_timing(apbf_scene *s, int enable)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    s->timing = enable != 0;
    return APBF_OK;
}

APBF_API apbf_status apbf_timing_report(apbf_scene *s, double *ms, uint64_t *launches)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (!ms || !launches)
        return fail(s, APBF_ERR_INVALID_ARG, "outputs are NULL");
    APBF_CUDA(s, cudaStreamSynchronize(s->stream));
    for (auto &t : s->timed) {
        float v = 0.0f;
        APBF_CUDA(s, cudaEventElapsedTime(&v, t.a, t.b));
        s->stage_ms[t.stage] += v;
        s->stage_launches[t.stage] += 1;
        s->ev_pool.push_back(t.a);
        s->ev_pool.push_back(t.b);
    }
    s->timed.clear();
    for (uint32_t k = 0; k < APBF_STAGE_COUNT; ++k) {
        ms[k] = s->stage_ms[k];
        launches[k] = s->stage_launches[k];
        s->stage_ms[k] = 0.0;
        s->stage_launches[k] = 0;
    }
    return APBF_OK;
}

}  // extern "C"

namespace apbf {
void drop_graph(apbf_scene *s)
{
    if (s->gexec)
        cudaGraphExecDestroy(s->gexec);
    if (s->graph)
        cudaGraphDestroy(s->graph);
    s->gexec = nullptr;
    s->graph = nullptr;
}
}  // namespace apbf

extern "C" {
namespace {
apbf_status copy_state(apbf_scene *s, bool to_snapshot)
{
    const Buffers &b = s->b;
    const size_t n = s->sc.n;
    float4 *x0 = to_snapshot ? b.snap_x : b.state_x, *x1 = to_snapshot ? b.state_x : b.snap_x;
    float4 *v0 = to_snapshot ? b.snap_v : b.state_v, *v1 = to_snapshot ? b.state_v : b.snap_v;
    uint32_t *i0 = to_snapshot ? b.snap_id : b.state_id, *i1 = to_snapshot ? b.state_id : b.snap_id;
    APBF_CUDA(s, cudaMemcpyAsync(x0, x1, 16 * n, cudaMemcpyDeviceToDevice, s->stream));
    APBF_CUDA(s, cudaMemcpyAsync(v0, v1, 16 * n, cudaMemcpyDeviceToDevice, s->stream));
    APBF_CUDA(s, cudaMemcpyAsync(i0, i1, 4 * n, cudaMemcpyDeviceToDevice, s->stream));
    return APBF_OK;
}
}  // namespace

APBF_API apbf_status apbf_set_tuning(apbf_scene *s, uint32_t block, float mask_threshold)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if ((block != 128 && block != 256) || !(mask_threshold >= 0.0f) || !std::isfinite(mask_threshold))
        return fail(s, APBF_ERR_INVALID_ARG, "block must be 128 or 256 and mask_threshold finite and >= 0");
    s->tune.block = (int)block;
    s->tune.mask_threshold = mask_threshold;
    drop_graph(s);
    return APBF_OK;
}

APBF_API apbf_status apbf_autotune(apbf_scene *s, uint32_t trial_steps, apbf_tune_result *out)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (!out || trial_steps == 0 || trial_steps > 1000)
        return fail(s, APBF_ERR_INVALID_ARG, "out is NULL or trial_steps not in 1..1000");
    if (s->sc.lod_mode == APBF_LOD_DTVS && !s->view_set)
        return fail(s, APBF_ERR_BAD_STATE, "a DTVS scene needs apbf_set_view before it steps");
    std::memset(out, 0, sizeof(*out));
    out->block = (uint32_t)s->tune.block;
    out->mask_threshold = s->tune.mask_threshold;
    if (s->sc.n == 0)
        return APBF_OK;
    const uint32_t blocks[2] = {256, 128};
    const float thresholds[5] = {2.0f, 0.9f, 0.75f, 0.5f, 0.0f};
    if ((st = upload_dyn(s)) != APBF_OK)
        return st;
    if ((st = copy_state(s, true)) != APBF_OK)
        return st;
    // the trial steps do not count in the running total of particle-iterations
    APBF_CUDA(s, cudaMemcpyAsync(s->b.counters + kIterSaveSlot, s->b.counters + kIterTotalSlot, 8,
                                 cudaMemcpyDeviceToDevice, s->stream));
    cudaEvent_t e0 = get_event(s), e1 = get_event(s);
    const bool timing = s->timing;
    s->timing = false;
    double best = 1e300;
    Tune best_t = s->tune;
    uint32_t k = 0;
    for (uint32_t bi = 0; bi < 2; ++bi)
        for (uint32_t ti = 0; ti < 5; ++ti, ++k) {
            s->tune.block = (int)blocks[bi];
            s->tune.mask_threshold = thresholds[ti];
            if ((st = copy_state(s, false)) != APBF_OK)
                break;
            for (uint32_t w = 0; w < 2 && st == APBF_OK; ++w)
                st = enqueue_step(s, s->stream, kStageAll, 0);
            if (st != APBF_OK)
                break;
            APBF_CUDA(s, cudaEventRecord(e0, s->stream));
            for (uint32_t w = 0; w < trial_steps && st == APBF_OK; ++w)
                st = enqueue_step(s, s->stream, kStageAll, 0);
            if (st != APBF_OK)
                break;
            APBF_CUDA(s, cudaEventRecord(e1, s->stream));
            APBF_CUDA(s, cudaEventSynchronize(e1));
            float ms = 0.0f;
            APBF_CUDA(s, cudaEventElapsedTime(&ms, e0, e1));
            const double per = (double)ms / trial_steps;
            out->ms[k] = per;
            out->blocks[k] = blocks[bi];
            out->thresholds[k] = thresholds[ti];
            if (per < best) {
                best = per;
                best_t = s->tune;
            }
        }
    s->timing = timing;
    s->ev_pool.push_back(e0);
    s->ev_pool.push_back(e1);
    if (st != APBF_OK)
        return st;
    out->tried = k;
    if ((st = copy_state(s, false)) != APBF_OK)
        return st;
    APBF_CUDA(s, cudaMemcpyAsync(s->b.counters + kIterTotalSlot, s->b.counters + kIterSaveSlot, 8,
                                 cudaMemcpyDeviceToDevice, s->stream));
    APBF_CUDA(s, cudaStreamSynchronize(s->stream));
    s->tune = best_t;
    drop_graph(s);
    out->block = (uint32_t)best_t.block;
    out->mask_threshold = best_t.mask_threshold;
    out->ms_per_step = best;
    return check_device_errors(s);
}

APBF_API apbf_status apbf_debug_step_to(apbf_scene *s, uint32_t stage, uint32_t iteration)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (stage >= APBF_STAGE_COUNT)
        return fail(s, APBF_ERR_INVALID_ARG, "unknown stage");
    if ((stage == APBF_STAGE_LAMBDA || stage == APBF_STAGE_DELTAP) && (iteration < 1 || iteration > s->sc.n_max))
        return fail(s, APBF_ERR_INVALID_ARG, "iteration must be in 1..n_max");
    if (s->sc.lod_mode == APBF_LOD_DTVS && !s->view_set)
        return fail(s, APBF_ERR_BAD_STATE, "a DTVS scene needs apbf_set_view before it steps");
    if (s->sc.n == 0)
        return APBF_OK;
    if ((st = upload_dyn(s)) != APBF_OK)
        return st;
    st = enqueue_step(s, s->stream, stage == APBF_STAGE_FINALIZE ? kStageAll : stage, iteration);
    if (st != APBF_OK)
        return st;
    if (stage < APBF_STAGE_SCAN)  // the scan, which clears the cell counts, did not run
        APBF_CUDA(s, cudaMemsetAsync(s->b.cnt, 0, 4 * (size_t)((s->sc.ncell + 3) / 4 * 4), s->stream));
    if (stage == APBF_STAGE_FINALIZE)
        s->stepped = true;
    APBF_CUDA(s, cudaStreamSynchronize(s->stream));
    return APBF_OK;
}

APBF_API apbf_status apbf_debug_read(apbf_scene *s, uint32_t field, void *host, size_t bytes)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    const StepConst &sc = s->sc;
    const Buffers &b = s->b;
    const size_t n = sc.n;
    const void *src = nullptr;
    size_t size = 0;
    const float4 *cur = s->cur_buf ? b.recB : b.recA;
    if (s->copy_pending)  // some fields are staged in the buffer an asynchronous readback may still copy
        APBF_CUDA(s, cudaStreamWaitEvent(s->stream, s->copy_ev, 0));
    switch (field) {
    case APBF_DBG_KEYS: src = b.key; size = 4 * n; break;
    case APBF_DBG_STATE_IDS: src = b.state_id; size = 4 * n; break;
    case APBF_DBG_LEVEL_PRESORT: src = b.lvl; size = n; break;
    case APBF_DBG_SORTED_IDS: src = b.id_s; size = 4 * n; break;
    case APBF_DBG_CELL_START: src = b.start; size = 4 * ((size_t)sc.ncell + 1); break;
    case APBF_DBG_XPRED: src = b.xs32; size = 16 * n; break;
    case APBF_DBG_LEVEL: src = b.lvl_s; size = n; break;
    case APBF_DBG_NBR_COUNT: src = b.nbr_cnt; size = n; break;
    case APBF_DBG_NBR: src = b.nbr; size = 4 * (size_t)sc.max_nbr * n; break;
    case APBF_DBG_ACTIVE: src = b.act; size = 4 * n; break;
    case APBF_DBG_LEVEL_COUNT: src = b.lvl_count; size = 4 * ((size_t)sc.n_max + 2); break;
    case APBF_DBG_LAMBDA:
        APBF_CUDA(s, launch_debug_lambda(sc, b, cur, s->stream));
        src = b.stage_f;
        size = 4 * n;
        break;
    case APBF_DBG_RHO: src = b.rho; size = 4 * n; break;
    case APBF_DBG_XSTAR:
        APBF_CUDA(s, launch_debug_xstar(sc, b, cur, s->stream));
        src = b.dbg4;
        size = 16 * n;
        break;
    case APBF_DBG_DRANGE: src = b.drange; size = 8 * (size_t)sc.scenes; break;
    case APBF_DBG_DEPTH:
        src = s->view.depth;
        size = s->view_set ? 4 * (size_t)s->view.W * s->view.H : 0;
        break;
    case APBF_DBG_LOD_DISTANCE: src = b.lodd; size = 4 * n; break;
    default: return fail(s, APBF_ERR_INVALID_ARG, "unknown debug field");
    }
    if (bytes != size || (size && !host))
        return fail(s, APBF_ERR_INVALID_ARG, "debug_read size mismatch: field needs " + std::to_string(size) + " bytes");
    if ((field == APBF_DBG_NBR || field == APBF_DBG_NBR_COUNT) && n && (field == APBF_DBG_NBR || !s->lists_by_slot)) {
        // stored in entry blocks by list column (the active-list position when
        // the step is partitioned): report entry k of sorted slot p at k*n + p
        std::vector<uint32_t> col(n);
        if (s->lists_by_slot) {
            for (size_t t = 0; t < n; ++t)
                col[t] = (uint32_t)t;
        } else {
            APBF_CUDA(s, cudaMemcpyAsync(col.data(), b.act, 4 * n, cudaMemcpyDeviceToHost, s->stream));
        }
        if (field == APBF_DBG_NBR_COUNT) {
            std::vector<uint8_t> raw(n);
            APBF_CUDA(s, cudaMemcpyAsync(raw.data(), b.nbr_cnt, n, cudaMemcpyDeviceToHost, s->stream));
            APBF_CUDA(s, cudaStreamSynchronize(s->stream));
            for (size_t t = 0; t < n; ++t)
                ((uint8_t *)host)[col[t]] = raw[t];
        } else {
            std::vector<uint32_t> raw((size_t)list_rows(sc.max_nbr) * n);
            APBF_CUDA(s, cudaMemcpyAsync(raw.data(), b.nbr, 4 * raw.size(), cudaMemcpyDeviceToHost, s->stream));
            APBF_CUDA(s, cudaStreamSynchronize(s->stream));
            for (uint32_t k = 0; k < sc.max_nbr; ++k)
                for (size_t t = 0; t < n; ++t)
                    ((uint32_t *)host)[k * n + col[t]] = raw[entry_index(k, t, n)];
        }
        return check_device_errors(s);
    }
    if (size)
        APBF_CUDA(s, cudaMemcpyAsync(host, src, size, cudaMemcpyDeviceToHost, s->stream));
    APBF_CUDA(s, cudaStreamSynchronize(s->stream));
    if (field == APBF_DBG_DRANGE)  // the minima are kept as the complements of their bit patterns
        for (uint32_t k = 0; k < sc.scenes; ++k)
            ((uint32_t *)host)[k] = ~((uint32_t *)host)[k];
    return check_device_errors(s);
}

APBF_API int apbf_debug_checks_enabled(void) { return APBF_DEBUG_CHECKS ? 1 : 0; }

APBF_API apbf_status apbf_debug_plant(apbf_scene *s, uint32_t what)
{
    apbf_status st = enter(s);
    if (st != APBF_OK)
        return st;
    if (!APBF_DEBUG_CHECKS)
        return fail(s, APBF_ERR_NOT_SUPPORTED, "apbf_debug_plant needs the debug build (libapbf_debug.so)");
    if (what > 1)
        return fail(s, APBF_ERR_INVALID_ARG, "what must be 0 or 1");
    APBF_CUDA(s, cudaMemcpyAsync(s->b.dbg + 2, &what, 4, cudaMemcpyHostToDevice, s->stream));
    APBF_CUDA(s, cudaStreamSynchronize(s->stream));
    return APBF_OK;
}

APBF_API apbf_status apbf_debug_dims(apbf_scene *s, int32_t dims[3], uint32_t *ncell, uint32_t *max_neighbors)
{
    if (!s || !dims || !ncell || !max_neighbors)
        return APBF_ERR_INVALID_ARG;
    dims[0] = s->sc.nx;
    dims[1] = s->sc.ny;
    dims[2] = s->sc.nz;
    *ncell = s->sc.ncell;
    *max_neighbors = s->sc.max_nbr;
    return APBF_OK;
}

}  // extern "C"
