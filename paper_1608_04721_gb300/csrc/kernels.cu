// CUDA kernels of one Adaptive Position-Based Fluids step (Fig. 7, Sec. 5),
// written for sm_103a. Host orchestration lives in apbf_capi.cu.
//
// Data layout (structure of arrays, sorted by cell after the reorder):
//   state_x, state_v  float4 per particle (w unused), the state between steps
//   recA / recB       float4 per particle: position relative to the particle's
//                     cell origin (xyz) and lambda (w); the two Jacobi buffers
//   xs32              float4 absolute predicted position (FP32), for the
//                     neighbour predicate
//   xt                float4 start-of-step position relative to the cell origin
//   nbr               u32 neighbour entries, entry k of particle p at k*n + p
//                     (a warp of consecutive particles reads one 128-byte line
//                     per k); low 27 bits: sorted slot, high 5 bits: which of
//                     the 27 neighbour cells the neighbour was found in.
//
// Positions inside the solver are stored relative to the particle's cell
// origin (m + c) * q, with q = h rounded to 8 significant bits so that every
// origin and every origin difference (+-q per axis) is exact in FP32. The
// difference of two positions is then (p_i - p_j) + dtab[code] with |p| ~ h,
// which keeps FP32 rounding at the scale of h instead of the scale of the
// domain (a 10 m basin has an FP32 spacing of ~1e-6 m).
#include "apbf_internal.h"

#include "device_common.cuh"

namespace apbf {
namespace {

// ------------------------------------------------------------- a1: range

__global__ void __launch_bounds__(kBlock) lod_range_kernel(StepConst sc, Buffers b)
{
    __shared__ float smin[kBlock / 32], smax[kBlock / 32];
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    float dmin = 3.0e38f, dmax = 0.0f;
    if (i < sc.n) {
        float d = camera_distance(b.state_x[i], b.dyn);
        dmin = d;
        dmax = d;
    }
    dmin = warp_minf(dmin);
    dmax = warp_maxf(dmax);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        smin[w] = dmin;
        smax[w] = dmax;
    }
    __syncthreads();
    if (w == 0) {
        dmin = lane < kBlock / 32 ? smin[lane] : 3.0e38f;
        dmax = lane < kBlock / 32 ? smax[lane] : 0.0f;
        dmin = warp_minf(dmin);
        dmax = warp_maxf(dmax);
        if (lane == 0) {
            // distances are >= 0, so their bit patterns order like the values
            atomicMin(&b.drange[0], __float_as_uint(dmin));
            atomicMax(&b.drange[1], __float_as_uint(dmax));
        }
    }
}

// ------------------------------------- a1-a4: level, predict, hash, count

__global__ void __launch_bounds__(kBlock) predict_hash_kernel(StepConst sc, Buffers b, int diag)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = i < sc.n;
    uint32_t key = 0xffffffffu;
    if (valid) {
        float4 x = b.state_x[i];
        float3 p;
        if (diag) {
            p = make_float3(x.x, x.y, x.z);
        } else {
            uint32_t lv = sc.n_max;
            if (sc.lod_mode == APBF_LOD_DTC) {
                const DynParams *dyn = b.dyn;
                float dmin = dyn->d_near, dmax = dyn->d_far;
                if (dyn->auto_range) {
                    dmin = __uint_as_float(b.drange[0]);
                    dmax = __uint_as_float(b.drange[1]);
                }
                lv = lod_level(camera_distance(x, dyn), dmin, dmax, sc);
            }
            b.lvl[i] = (uint8_t)lv;
            p = predict_position(x, b.state_v[i], sc, b.dyn);
        }
        int3 c = cell_of(p, sc);
        key = ((uint32_t)c.z * (uint32_t)sc.ny + (uint32_t)c.y) * (uint32_t)sc.nx + (uint32_t)c.x;
        b.key[i] = key;
    }
    // warp-aggregated histogram: one atomic per distinct cell in the warp
    unsigned peers = __match_any_sync(kFull, key);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (valid && lane == leader)
        base = atomicAdd(&b.cnt[key], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    if (valid)
        b.slot[i] = base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
}

// ------------------------------------------------ a4/a6: scan = cell start

__global__ void __launch_bounds__(1024) scan_reduce_kernel(const uint32_t *__restrict__ cnt, uint32_t ncell,
                                                           uint32_t *__restrict__ tile_sums)
{
    __shared__ uint32_t sh[32];
    uint32_t base = blockIdx.x * kScanTile + threadIdx.x * 4;
    uint32_t s = 0;
    if (base + 3 < ncell) {
        uint4 v = *reinterpret_cast<const uint4 *>(cnt + base);
        s = v.x + v.y + v.z + v.w;
    } else {
        for (uint32_t k = base; k < ncell && k < base + 4; ++k)
            s += cnt[k];
    }
    s = block_sum_u32(s, sh);
    if (threadIdx.x == 0)
        tile_sums[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) scan_apply_kernel(uint32_t *__restrict__ cnt, uint32_t ncell,
                                                          const uint32_t *__restrict__ tile_sums,
                                                          uint32_t *__restrict__ start, uint32_t n)
{
    __shared__ uint32_t sh[32];
    uint32_t pre = 0;
    for (uint32_t t = threadIdx.x; t < blockIdx.x; t += blockDim.x)
        pre += tile_sums[t];
    pre = block_sum_u32(pre, sh);
    uint32_t base = blockIdx.x * kScanTile + threadIdx.x * 4;
    uint32_t v[4] = {0u, 0u, 0u, 0u};
    if (base + 3 < ncell) {
        uint4 q = *reinterpret_cast<const uint4 *>(cnt + base);
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
        *reinterpret_cast<uint4 *>(cnt + base) = make_uint4(0u, 0u, 0u, 0u);  // ready for the next step
    } else {
        for (uint32_t k = 0; k < 4; ++k)
            if (base + k < ncell) {
                v[k] = cnt[base + k];
                cnt[base + k] = 0u;
            }
    }
    uint32_t total;
    uint32_t ex = block_exclusive_scan_u32(v[0] + v[1] + v[2] + v[3], sh, &total);
    uint32_t run = pre + ex;
    for (uint32_t k = 0; k < 4; ++k) {
        if (base + k < ncell)
            start[base + k] = run;
        run += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        start[ncell] = n;
}

// ------------------------------------------ a4: slot scatter (particle ids)

__global__ void __launch_bounds__(kBlock) scatter_kernel(StepConst sc, Buffers b)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < sc.n)
        b.tmp[b.start[b.key[i]] + b.slot[i]] = b.state_id[i];
}

// ------------------------------------------ a4/a5: stable rank + reorder

__global__ void __launch_bounds__(kBlock) reorder_kernel(StepConst sc, Buffers b, int diag)
{
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sc.n)
        return;
    uint32_t k = b.key[i];
    uint32_t s0 = b.start[k], s1 = b.start[k + 1];
    // order within a cell by particle id: rank = number of this cell's
    // particles with a smaller id (the slots hold ids in atomic arrival order)
    const uint32_t id = b.state_id[i];
    uint32_t r = 0;
    for (uint32_t j = s0; j < s1; ++j)
        r += (b.tmp[j] < id) ? 1u : 0u;
    uint32_t p = s0 + r;
    float4 x = b.state_x[i];
    float3 xp = diag ? make_float3(x.x, x.y, x.z) : predict_position(x, b.state_v[i], sc, b.dyn);
    int3 c = cell_of(xp, sc);
    b.xs32[p] = make_float4(xp.x, xp.y, xp.z, 0.0f);
    b.cell_s[p] = pack_cell(c);
    if (!diag) {
        float3 o = cell_origin(c, sc);
        b.recA[p] = make_float4(__fsub_rn(xp.x, o.x), __fsub_rn(xp.y, o.y), __fsub_rn(xp.z, o.z), 0.0f);
        b.xt[p] = make_float4(__fsub_rn(x.x, o.x), __fsub_rn(x.y, o.y), __fsub_rn(x.z, o.z), 0.0f);
        b.id_s[p] = id;
        b.lvl_s[p] = b.lvl[i];
    }
}

// ------------------------------------------------------- readback helpers

__global__ void __launch_bounds__(kBlock) unpermute_kernel(StepConst sc, Buffers b, uint32_t what)
{
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= sc.n)
        return;
    uint32_t id = b.state_id[p];
    if (what == 0 || what == 1) {
        float4 v = (what == 0) ? b.state_x[p] : b.state_v[p];
        b.stage_f[3 * (size_t)id + 0] = v.x;
        b.stage_f[3 * (size_t)id + 1] = v.y;
        b.stage_f[3 * (size_t)id + 2] = v.z;
    } else if (what == 2) {
        b.stage_u8[id] = b.lvl_s[p];
    } else {
        b.stage_f[id] = b.rho[p];
    }
}

__global__ void __launch_bounds__(32) density_final_kernel(const double *__restrict__ partials, int nblocks,
                                                           uint32_t n, double *__restrict__ out)
{
    // one warp, fixed summation order
    double a = 0, m = 0, s = 0, q = 0;
    for (int k = threadIdx.x; k < nblocks; k += 32) {
        a += partials[4 * k + 0];
        m = fmax(m, partials[4 * k + 1]);
        s += partials[4 * k + 2];
        q += partials[4 * k + 3];
    }
    a = warp_sum(a);
    s = warp_sum(s);
    q = warp_sum(q);
    m = warp_max(m);
    if (threadIdx.x == 0) {
        out[0] = n ? a / n : 0.0;
        out[1] = m;
        out[2] = n ? s / n : 0.0;
        out[3] = n ? q / n : 0.0;
    }
}

__global__ void __launch_bounds__(kBlock) debug_xstar_kernel(StepConst sc, Buffers b, const float4 *__restrict__ rec)
{
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= sc.n)
        return;
    const float4 r = rec[p];
    const float3 og = cell_origin(unpack_cell(b.cell_s[p]), sc);
    b.dbg4[p] = make_float4(og.x + r.x, og.y + r.y, og.z + r.z, 0.0f);
}

__global__ void __launch_bounds__(kBlock) debug_lambda_kernel(StepConst sc, Buffers b, const float4 *__restrict__ rec)
{
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < sc.n)
        b.stage_f[p] = rec[p].w;
}

inline unsigned blocks_for(uint32_t n, int bs) { return (unsigned)((n + (uint32_t)bs - 1) / (uint32_t)bs); }

}  // namespace

// ------------------------------------------------------------- launchers

// Resident blocks per SM of a kernel launched with `block` threads (cached per function).
int occupancy(const void *fn, int block)
{
    static const void *keys[16];
    static int vals[16];
    for (int k = 0; k < 16; ++k)
        if (keys[k] == fn)
            return vals[k];
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, 0) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 4;
    }
    for (int k = 0; k < 16; ++k)
        if (!keys[k]) {
            keys[k] = fn;
            vals[k] = occ;
            break;
        }
    return occ;
}


cudaError_t launch_lod_range(const StepConst &sc, const Buffers &b, cudaStream_t s)
{
    if (sc.n)
        lod_range_kernel<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc, b);
    return cudaGetLastError();
}

cudaError_t launch_predict_hash(const StepConst &sc, const Buffers &b, cudaStream_t s, bool diag)
{
    if (sc.n)
        predict_hash_kernel<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc, b, diag ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_scan(const StepConst &sc, const Buffers &b, cudaStream_t s)
{
    unsigned tiles = blocks_for(sc.ncell, kScanTile);
    scan_reduce_kernel<<<tiles, 1024, 0, s>>>(b.cnt, sc.ncell, b.tile_sums);
    scan_apply_kernel<<<tiles, 1024, 0, s>>>(b.cnt, sc.ncell, b.tile_sums, b.start, sc.n);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const StepConst &sc, const Buffers &b, cudaStream_t s)
{
    if (sc.n)
        scatter_kernel<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc, b);
    return cudaGetLastError();
}

cudaError_t launch_reorder(const StepConst &sc, const Buffers &b, cudaStream_t s, bool diag)
{
    if (sc.n)
        reorder_kernel<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc, b, diag ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_unpermute(const StepConst &sc, const Buffers &b, cudaStream_t s, uint32_t what)
{
    if (sc.n)
        unpermute_kernel<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc, b, what);
    return cudaGetLastError();
}

cudaError_t launch_density_final(const StepConst &sc, const Buffers &b, cudaStream_t s, int nblocks)
{
    density_final_kernel<<<1, 32, 0, s>>>(b.partials, nblocks, sc.n, b.dstats);
    return cudaGetLastError();
}

cudaError_t launch_debug_xstar(const StepConst &sc, const Buffers &b, const float4 *rec, cudaStream_t s)
{
    if (sc.n)
        debug_xstar_kernel<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc, b, rec);
    return cudaGetLastError();
}

cudaError_t launch_debug_lambda(const StepConst &sc, const Buffers &b, const float4 *rec, cudaStream_t s)
{
    if (sc.n)
        debug_lambda_kernel<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc, b, rec);
    return cudaGetLastError();
}


}  // namespace apbf
