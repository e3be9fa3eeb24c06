// Tile-staged kernels of one Adaptive Position-Based Fluids step for sm_103a:
// neighbour lists (Fig. 7 lines 5-6), the active-set partition (Eq. 9-11),
// the lambda pass (Eq. 4-6, Fig. 7 lines 13-15), the position-correction pass
// with contacts and the Jacobi update (Eq. 7, lines 16-22), the velocity /
// XSPH commit (lines 24-27) and the density diagnostic (Fig. 9).
//
// Work unit: a tile = kTileX consecutive cells of one grid row (y, z).
// Particles are sorted by cell key (z, y, x), so a tile's particles are a
// contiguous slot range and all their neighbours lie in 9 contiguous "runs":
// rows (y+dy, z+dz), dy, dz in {-1, 0, 1}, cells x0-1 .. x1. A persistent CTA
// takes tiles in turn; one elected thread copies the runs into shared memory
// with bulk asynchronous copies (cp.async.bulk, the TMA engine) that complete
// on an mbarrier, and then every thread handles one particle of the tile with
// all neighbour reads served from shared memory. A tile whose halo exceeds
// kTileCap records is processed from global memory by the same code.
//
// Neighbour entries are 16 bits: the cell offset code (which of the 27 cells)
// and the neighbour's offset within its run; the run's base (in shared or in
// global memory) comes from a per-tile 27-entry table that also holds the
// cell-origin difference of that code.
#include "device_common.cuh"

namespace apbf {
namespace {

struct TileRuns {
    uint32_t slot0[9];  // first particle slot of each run
    uint32_t len[9];    // particles in each run
    uint32_t base[9];   // position of each run in the staged buffer
    int xa[9];          // first cell x of each run
    uint32_t total;     // records of all runs
    uint32_t p0, p1;    // the tile's own particles
    int x0, x1, xb, cy, cz;
};

constexpr uint32_t kWaitTries = 1u << 20;

// ------------------------------------------ bulk copies on an mbarrier (TMA)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Bounded wait for the mbarrier phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (uint32_t it = 0; it < kWaitTries; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.b32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done)
            return true;
    }
    return false;
}

// Copy the tile's runs of `src` into `dst`. Returns false in every thread
// when the copies did not complete within the bounded waits (error flagged).
__device__ bool stage_tile(const TileRuns &g, const float4 *__restrict__ src, float4 *dst, uint64_t *bar,
                           uint32_t &phase, uint32_t *err)
{
    if (threadIdx.x == 0) {
        // the CTA's earlier reads of dst (ordered by the preceding barrier)
        // happen before the asynchronous writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                     "r"(g.total * 16u)
                     : "memory");
        for (int r = 0; r < 9; ++r)
            if (g.len[r])
                bulk_copy_g2s(dst + g.base[r], src + g.slot0[r], g.len[r] * 16u, bar);
    }
    bool ok = mbar_wait(bar, phase);
    if (!ok)
        ok = mbar_wait(bar, phase);  // a second bounded wait for copies still in flight
    phase ^= 1u;
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0)
            atomicOr(err, kErrTimeout);
        return false;
    }
    return true;
}

// Geometry of tile t (cells x0..x1-1 of row (cy, cz)) and its 9 halo runs.
__device__ void tile_geometry(const StepConst &sc, const uint32_t *__restrict__ start, uint32_t t, TileRuns &g)
{
    __syncthreads();  // previous readers of g are done
    const uint32_t row = t / sc.tiles_per_row;
    const int seg = (int)(t - row * sc.tiles_per_row);
    const int cy = (int)(row % (uint32_t)sc.ny), cz = (int)(row / (uint32_t)sc.ny);
    const int x0 = seg * kTileX, x1 = min(x0 + kTileX, sc.nx), xa = max(x0 - 1, 0), xb = min(x1 + 1, sc.nx);
    if (threadIdx.x < 9) {
        const int r = threadIdx.x, yy = cy + r % 3 - 1, zz = cz + r / 3 - 1;
        uint32_t s0 = 0, s1 = 0;
        if (yy >= 0 && yy < sc.ny && zz >= 0 && zz < sc.nz) {
            const uint32_t rb = ((uint32_t)zz * (uint32_t)sc.ny + (uint32_t)yy) * (uint32_t)sc.nx;
            s0 = start[rb + xa];
            s1 = start[rb + xb];
        }
        g.slot0[r] = s0;
        g.len[r] = s1 - s0;
        g.xa[r] = xa;
    } else if (threadIdx.x == 32) {
        const uint32_t rb = row * (uint32_t)sc.nx;
        g.p0 = start[rb + x0];
        g.p1 = start[rb + x1];
        g.x0 = x0;
        g.x1 = x1;
        g.xb = xb;
        g.cy = cy;
        g.cz = cz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int r = 0; r < 9; ++r) {
            g.base[r] = acc;
            acc += g.len[r];
        }
        g.total = acc;
    }
    __syncthreads();
}

// code -> (cell-origin difference o_i - o_j, base index of the code's run)
__device__ __forceinline__ void fill_tile_dtab(float4 *dtab, const TileRuns &g, float q, bool staged)
{
    if (threadIdx.x < 27) {
        const int c = threadIdx.x, r = c / 3;
        const float ox = (float)(c % 3 - 1), oy = (float)((c / 3) % 3 - 1), oz = (float)(c / 9 - 1);
        dtab[c] = make_float4(-ox * q, -oy * q, -oz * q, __uint_as_float(staged ? g.base[r] : g.slot0[r]));
    }
}

constexpr int kBatch = 4;

// Visit particle p's neighbours in batches: the batch's 16-bit entries are
// loaded (coalesced across the warp) before its records are read.
template <typename F>
__device__ __forceinline__ void for_each_entry(const uint16_t *__restrict__ nbr, size_t n, uint32_t p, uint32_t nn,
                                               F &&f)
{
    for (uint32_t k = 0; k < nn; k += kBatch) {
        uint32_t e[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
            e[u] = (k + u < nn) ? (uint32_t)__ldg(nbr + (size_t)(k + u) * n + p) : 0xffffffffu;
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
            if (e[u] != 0xffffffffu)
                f(e[u]);
    }
}

// ------------------------------------------------ a7: levels and tile lists

__global__ void __launch_bounds__(256) tile_level_kernel(StepConst sc, Buffers b)
{
    const uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= sc.ntiles)
        return;  // warp-uniform
    const uint32_t row = t / sc.tiles_per_row;
    const int x0 = (int)(t - row * sc.tiles_per_row) * kTileX, x1 = min(x0 + kTileX, sc.nx);
    const uint32_t rb = row * (uint32_t)sc.nx;
    const uint32_t p0 = b.start[rb + x0], p1 = b.start[rb + x1];
    uint32_t m = 0;
    for (uint32_t p = p0 + lane; p < p1; p += 32)
        m = max(m, (uint32_t)b.lvl_s[p]);
    m = __reduce_max_sync(kFull, m);
    if (lane == 0)
        b.tile_lvl[t] = (uint8_t)m;
}

// Stable partition of `count` values by bin = vmax - value (highest value first).
struct PartArgs {
    const uint8_t *val;
    const uint8_t *weight;  // optional, summed per bin into wsum
    uint32_t count, vmax, nbins, blocks;
    uint32_t *hist, *off, *list, *count_ge;
    unsigned long long *wsum;
};

__global__ void __launch_bounds__(kPartBlock) part_hist_kernel(PartArgs a)
{
    extern __shared__ uint32_t sh[];  // nbins counts, nbins weights
    for (uint32_t k = threadIdx.x; k < 2 * a.nbins; k += blockDim.x)
        sh[k] = 0u;
    __syncthreads();
    const uint32_t i = blockIdx.x * kPartBlock + threadIdx.x;
    if (i < a.count) {
        const uint32_t bin = a.vmax - a.val[i];
        atomicAdd(&sh[bin], 1u);
        if (a.weight)
            atomicAdd(&sh[a.nbins + bin], (uint32_t)a.weight[i]);
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < a.nbins; k += blockDim.x) {
        a.hist[(size_t)k * a.blocks + blockIdx.x] = sh[k];
        if (a.weight && sh[a.nbins + k])
            atomicAdd(&a.wsum[k], (unsigned long long)sh[a.nbins + k]);
    }
}

__global__ void __launch_bounds__(1024) part_scan_kernel(PartArgs a)
{
    __shared__ uint32_t sh[32];
    const uint32_t E = a.nbins * a.blocks;
    const uint32_t chunk = (E + blockDim.x - 1) / blockDim.x;
    const uint32_t e0 = min(E, threadIdx.x * chunk), e1 = min(E, e0 + chunk);
    uint32_t s = 0;
    for (uint32_t e = e0; e < e1; ++e)
        s += a.hist[e];
    uint32_t total;
    uint32_t run = block_exclusive_scan_u32(s, sh, &total);
    for (uint32_t e = e0; e < e1; ++e) {
        const uint32_t v = a.hist[e];
        a.off[e] = run;
        run += v;
    }
    __syncthreads();
    for (uint32_t l = threadIdx.x; l <= a.vmax + 1; l += blockDim.x) {
        uint32_t c;
        if (l > a.vmax)
            c = 0;
        else {
            const uint32_t bin_end = a.vmax - l + 1;  // bins 0 .. vmax-l hold values >= l
            c = (bin_end >= a.nbins) ? a.count : a.off[(size_t)bin_end * a.blocks];
        }
        a.count_ge[l] = c;
    }
}

__global__ void __launch_bounds__(kPartBlock) part_scatter_kernel(PartArgs a)
{
    extern __shared__ uint32_t wc[];  // 32 warps x nbins
    for (uint32_t k = threadIdx.x; k < 32 * a.nbins; k += blockDim.x)
        wc[k] = 0u;
    __syncthreads();
    const uint32_t i = blockIdx.x * kPartBlock + threadIdx.x;
    const bool valid = i < a.count;
    const uint32_t bin = valid ? (a.vmax - a.val[i]) : 0xffffffffu;
    const unsigned peers = __match_any_sync(kFull, bin);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int leader = __ffs(peers) - 1;
    const uint32_t rank = (uint32_t)__popc(peers & ((1u << lane) - 1u));
    if (valid && lane == leader)
        wc[w * a.nbins + bin] = (uint32_t)__popc(peers);
    __syncthreads();
    if (valid) {
        uint32_t pos = a.off[(size_t)bin * a.blocks + blockIdx.x] + rank;
        for (int v = 0; v < w; ++v)
            pos += wc[v * a.nbins + bin];
        a.list[pos] = i;
    }
}

// ------------------------------------------- neighbour lists (l. 5-6)
// Predicate on the FP32 predicted positions (absolute), rounded after every
// operation, exactly as the oracle defines it.

__global__ void __launch_bounds__(kTileThreads) neighbors_tile_kernel(StepConst sc, Buffers b)
{
    __shared__ __align__(128) float4 srec[kTileCap];
    __shared__ TileRuns g;
    __shared__ uint32_t cs[9][kTileX + 3];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t red[32];
    if (threadIdx.x == 0)
        mbar_init(&bar);
    __syncthreads();
    uint32_t phase = 0, pairs = 0;
    const size_t n = sc.n;
    for (uint32_t t = blockIdx.x; t < sc.ntiles; t += gridDim.x) {
        tile_geometry(sc, b.start, t, g);
        if (g.p0 == g.p1)
            continue;
        const int ncs = g.xb - g.xa[4] + 1;  // cell starts per run
        for (int i = threadIdx.x; i < 9 * ncs; i += blockDim.x) {
            const int r = i / ncs, k = i - r * ncs;
            const int yy = g.cy + r % 3 - 1, zz = g.cz + r / 3 - 1;
            uint32_t v = 0;
            if (yy >= 0 && yy < sc.ny && zz >= 0 && zz < sc.nz)
                v = b.start[((uint32_t)zz * (uint32_t)sc.ny + (uint32_t)yy) * (uint32_t)sc.nx + g.xa[r] + k];
            cs[r][k] = v;
        }
        const bool staged = g.total <= kTileCap;
        if (staged && !stage_tile(g, b.xs32, srec, &bar, phase, b.err))
            return;
        __syncthreads();
        for (uint32_t p = g.p0 + threadIdx.x; p < g.p1; p += blockDim.x) {
            const float4 xi = staged ? srec[g.base[4] + (p - g.slot0[4])] : b.xs32[p];
            const int cx = unpack_cell(b.cell_s[p]).x;
            uint32_t cnt = 0, run_over = 0;
            for (int r = 0; r < 9; ++r) {
                if (!g.len[r])
                    continue;
                const uint32_t s0 = g.slot0[r];
                for (int dx = -1; dx <= 1; ++dx) {
                    const int c = cx + dx;
                    if (c < 0 || c >= sc.nx)
                        continue;
                    const int k = c - g.xa[r];
                    const uint32_t o0 = cs[r][k] - s0, o1 = cs[r][k + 1] - s0;
                    const uint32_t code = (uint32_t)((dx + 1) + 3 * r) << kOffBits;
                    for (uint32_t o = o0; o < o1; ++o) {
                        if (s0 + o == p)
                            continue;
                        const float4 xj = staged ? srec[g.base[r] + o] : b.xs32[s0 + o];
                        const float ddx = __fsub_rn(xi.x, xj.x);
                        const float ddy = __fsub_rn(xi.y, xj.y);
                        const float ddz = __fsub_rn(xi.z, xj.z);
                        float r2 = __fadd_rn(__fmul_rn(ddx, ddx), __fmul_rn(ddy, ddy));
                        r2 = __fadd_rn(r2, __fmul_rn(ddz, ddz));
                        if (r2 < sc.h2) {
                            if (cnt < sc.max_nbr)
                                b.nbr[(size_t)cnt * n + p] = (uint16_t)(code | (o & kOffMask));
                            run_over |= o >> kOffBits;
                            ++cnt;
                        }
                    }
                }
            }
            if (cnt > sc.max_nbr) {
                atomicOr(b.err, kErrNeighborOverflow);
                cnt = sc.max_nbr;
            }
            if (run_over)
                atomicOr(b.err, kErrRunOverflow);
            b.nbr_cnt[p] = (uint8_t)cnt;
            pairs += cnt;
        }
    }
    __syncthreads();
    const uint32_t tot = block_sum_u32(pairs, red);
    if (threadIdx.x == 0 && tot)
        atomicAdd(&b.counters[0], (unsigned long long)tot);
}

// --------------------------------------------------------- a8: lambda pass
// Iteration l over the tiles holding particles of level >= l-1: particles of
// P_l compute rho and lambda (Eq. 4-6) from A and write (position, lambda) to
// B; particles that finished in iteration l-1 copy their final position into
// B and keep their lambda there, so inactive neighbours enter Eq. 7 with
// their last lambda.

template <bool STAGED>
__device__ __forceinline__ void lambda_tile(const StepConst &sc, const TileRuns &g, const float4 *dtab,
                                            const float4 *rec, float4 *__restrict__ B, float *__restrict__ rho_out,
                                            const uint16_t *__restrict__ nbr, const uint8_t *__restrict__ nbr_cnt,
                                            const uint8_t *__restrict__ lvl_s, uint32_t l)
{
    const size_t n = sc.n;
    for (uint32_t p = g.p0 + threadIdx.x; p < g.p1; p += blockDim.x) {
        const uint32_t lv = lvl_s[p];
        if (lv + 1 < l)
            continue;
        const float4 ai = rec[(STAGED ? g.base[4] : g.slot0[4]) + (p - g.slot0[4])];
        if (lv < l) {
            B[p] = make_float4(ai.x, ai.y, ai.z, B[p].w);
            continue;
        }
        float racc = 0.0f, gx = 0.0f, gy = 0.0f, gz = 0.0f, s2 = 0.0f;
        for_each_entry(nbr, n, p, nbr_cnt[p], [&](uint32_t e) {
            const float4 o = dtab[e >> kOffBits];
            const float4 aj = rec[__float_as_uint(o.w) + (e & kOffMask)];
            const float dx = (ai.x - aj.x) + o.x;
            const float dy = (ai.y - aj.y) + o.y;
            const float dz = (ai.z - aj.z) + o.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < sc.h2) {
                const float u = sc.h2 - r2;
                racc += u * u * u;
                if (r2 > 0.0f) {
                    const float ir = rsqrtf(r2);
                    const float hr = sc.h - r2 * ir;
                    const float gw = hr * hr * ir;  // |grad W| / (45/(pi h^6)) / r
                    gx += gw * dx;
                    gy += gw * dy;
                    gz += gw * dz;
                    s2 += gw * gw * r2;
                }
            }
        });
        const float rho = sc.mass_poly6 * (sc.h6 + racc);
        const float C = rho * sc.inv_rho0 - 1.0f;
        const float denom = sc.c_lam * (gx * gx + gy * gy + gz * gz + s2) + sc.eps;
        B[p] = make_float4(ai.x, ai.y, ai.z, -C / denom);
        rho_out[p] = rho;
    }
}

__global__ void __launch_bounds__(kTileThreads) lambda_tile_kernel(StepConst sc, Buffers b, uint32_t l)
{
    __shared__ __align__(128) float4 srec[kTileCap];
    __shared__ TileRuns g;
    __shared__ float4 dtab[27];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0)
        mbar_init(&bar);
    __syncthreads();
    uint32_t phase = 0;
    const uint32_t ntl = b.tile_count[l > 1 ? l - 1 : 1];
    for (uint32_t ti = blockIdx.x; ti < ntl; ti += gridDim.x) {
        tile_geometry(sc, b.start, b.tile_list[ti], g);
        const bool staged = g.total <= kTileCap;
        if (staged && !stage_tile(g, b.recA, srec, &bar, phase, b.err))
            return;
        fill_tile_dtab(dtab, g, sc.q, staged);
        __syncthreads();
        if (staged)
            lambda_tile<true>(sc, g, dtab, srec, b.recB, b.rho, b.nbr, b.nbr_cnt, b.lvl_s, l);
        else
            lambda_tile<false>(sc, g, dtab, b.recA, b.recB, b.rho, b.nbr, b.nbr_cnt, b.lvl_s, l);
    }
}

// ------------------------------------------- a9: position correction pass
// Iteration l over the tiles holding P_l: Eq. 7 with the tensile term from B,
// the box contact, and the Jacobi update written to A.

template <int NPOW>
__device__ __forceinline__ float powi(float x, uint32_t n)
{
    if (NPOW == 4) {
        const float x2 = x * x;
        return x2 * x2;
    }
    float r = 1.0f;
    for (uint32_t e = 0; e < n; ++e)
        r *= x;
    return r;
}

template <bool STAGED, int NPOW>
__device__ __forceinline__ void deltap_tile(const StepConst &sc, const TileRuns &g, const float4 *dtab,
                                            const float4 *rec, float4 *__restrict__ A,
                                            const uint16_t *__restrict__ nbr, const uint8_t *__restrict__ nbr_cnt,
                                            const uint8_t *__restrict__ lvl_s, const uint32_t *__restrict__ cell_s,
                                            const float *box, uint32_t l)
{
    const size_t n = sc.n;
    for (uint32_t p = g.p0 + threadIdx.x; p < g.p1; p += blockDim.x) {
        if (lvl_s[p] < l)
            continue;
        const float4 bi = rec[(STAGED ? g.base[4] : g.slot0[4]) + (p - g.slot0[4])];
        float ax = 0.0f, ay = 0.0f, az = 0.0f;
        for_each_entry(nbr, n, p, nbr_cnt[p], [&](uint32_t e) {
            const float4 o = dtab[e >> kOffBits];
            const float4 bj = rec[__float_as_uint(o.w) + (e & kOffMask)];
            const float dx = (bi.x - bj.x) + o.x;
            const float dy = (bi.y - bj.y) + o.y;
            const float dz = (bi.z - bj.z) + o.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < sc.h2 && r2 > 0.0f) {
                const float ir = rsqrtf(r2);
                const float hr = sc.h - r2 * ir;
                const float gw = hr * hr * ir;
                const float u = (sc.h2 - r2) * sc.inv_wdq;  // W(r) / W(dq) = u^3
                const float scorr = sc.neg_k * powi<NPOW>(u * u * u, sc.scorr_n);
                const float f = (bi.w + bj.w + scorr) * gw;
                ax += f * dx;
                ay += f * dy;
                az += f * dz;
            }
        });
        // new position, clamped to the box expressed relative to the cell origin
        const float3 og = cell_origin(unpack_cell(cell_s[p]), sc);
        float px = bi.x + sc.c_dp * ax;
        float py = bi.y + sc.c_dp * ay;
        float pz = bi.z + sc.c_dp * az;
        px = fminf(fmaxf(px, box[0] - og.x), box[4] - og.x);
        py = fminf(fmaxf(py, box[1] - og.y), box[5] - og.y);
        pz = fminf(fmaxf(pz, box[2] - og.z), box[6] - og.z);
        A[p] = make_float4(px, py, pz, bi.w);
    }
}

template <int NPOW>
__global__ void __launch_bounds__(kTileThreads) deltap_tile_kernel(StepConst sc, Buffers b, uint32_t l)
{
    __shared__ __align__(128) float4 srec[kTileCap];
    __shared__ TileRuns g;
    __shared__ float4 dtab[27];
    __shared__ __align__(8) uint64_t bar;
    __shared__ float box[8];
    if (threadIdx.x == 0)
        mbar_init(&bar);
    if (threadIdx.x < 8)
        box[threadIdx.x] = threadIdx.x < 4 ? b.dyn->box_lo[threadIdx.x] : b.dyn->box_hi[threadIdx.x - 4];
    __syncthreads();
    uint32_t phase = 0;
    const uint32_t ntl = b.tile_count[l];
    for (uint32_t ti = blockIdx.x; ti < ntl; ti += gridDim.x) {
        tile_geometry(sc, b.start, b.tile_list[ti], g);
        const bool staged = g.total <= kTileCap;
        if (staged && !stage_tile(g, b.recB, srec, &bar, phase, b.err))
            return;
        fill_tile_dtab(dtab, g, sc.q, staged);
        __syncthreads();
        if (staged)
            deltap_tile<true, NPOW>(sc, g, dtab, srec, b.recA, b.nbr, b.nbr_cnt, b.lvl_s, b.cell_s, box, l);
        else
            deltap_tile<false, NPOW>(sc, g, dtab, b.recB, b.recA, b.nbr, b.nbr_cnt, b.lvl_s, b.cell_s, box, l);
    }
}

// ------------------------------------------ a10: velocity, XSPH, commit

template <bool STAGED>
__device__ __forceinline__ void finalize_tile(const StepConst &sc, const TileRuns &g, const float4 *dtab,
                                              const float4 *rec, const Buffers &b, const float *box)
{
    const size_t n = sc.n;
    for (uint32_t p = g.p0 + threadIdx.x; p < g.p1; p += blockDim.x) {
        const float4 af = rec[(STAGED ? g.base[4] : g.slot0[4]) + (p - g.slot0[4])];
        const float4 x0 = b.xt[p];
        const float vx = (af.x - x0.x) * sc.inv_dt;
        const float vy = (af.y - x0.y) * sc.inv_dt;
        const float vz = (af.z - x0.z) * sc.inv_dt;
        float sx = 0.0f, sy = 0.0f, sz = 0.0f;
        for_each_entry(b.nbr, n, p, b.nbr_cnt[p], [&](uint32_t e) {
            const uint32_t code = e >> kOffBits, off = e & kOffMask;
            const float4 o = dtab[code];
            const float4 aj = rec[__float_as_uint(o.w) + off];
            const float dx = (af.x - aj.x) + o.x;
            const float dy = (af.y - aj.y) + o.y;
            const float dz = (af.z - aj.z) + o.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < sc.h2) {
                const float w = sc.h2 - r2;
                const float W = w * w * w;
                const float4 xj = __ldg(&b.xt[g.slot0[code / 3] + off]);
                sx += ((aj.x - xj.x) * sc.inv_dt - vx) * W;
                sy += ((aj.y - xj.y) * sc.inv_dt - vy) * W;
                sz += ((aj.z - xj.z) * sc.inv_dt - vz) * W;
            }
        });
        const float3 og = cell_origin(unpack_cell(b.cell_s[p]), sc);
        const float px = fminf(fmaxf(og.x + af.x, box[0]), box[4]);
        const float py = fminf(fmaxf(og.y + af.y, box[1]), box[5]);
        const float pz = fminf(fmaxf(og.z + af.z, box[2]), box[6]);
        b.state_x[p] = make_float4(px, py, pz, 0.0f);
        b.state_v[p] = make_float4(vx + sc.c_xsph * sx, vy + sc.c_xsph * sy, vz + sc.c_xsph * sz, 0.0f);
        b.state_id[p] = b.id_s[p];
    }
}

__global__ void __launch_bounds__(kTileThreads) finalize_tile_kernel(StepConst sc, Buffers b)
{
    __shared__ __align__(128) float4 srec[kTileCap];
    __shared__ TileRuns g;
    __shared__ float4 dtab[27];
    __shared__ __align__(8) uint64_t bar;
    __shared__ float box[8];
    if (threadIdx.x == 0)
        mbar_init(&bar);
    if (threadIdx.x < 8)
        box[threadIdx.x] = threadIdx.x < 4 ? b.dyn->box_lo[threadIdx.x] : b.dyn->box_hi[threadIdx.x - 4];
    __syncthreads();
    uint32_t phase = 0;
    const uint32_t ntl = b.tile_count[1];
    for (uint32_t ti = blockIdx.x; ti < ntl; ti += gridDim.x) {
        tile_geometry(sc, b.start, b.tile_list[ti], g);
        const bool staged = g.total <= kTileCap;
        if (staged && !stage_tile(g, b.recA, srec, &bar, phase, b.err))
            return;
        fill_tile_dtab(dtab, g, sc.q, staged);
        __syncthreads();
        if (staged)
            finalize_tile<true>(sc, g, dtab, srec, b, box);
        else
            finalize_tile<false>(sc, g, dtab, b.recA, b, box);
    }
}

// ------------------------------- density diagnostic (Fig. 9), FP64 partials

__global__ void __launch_bounds__(kTileThreads) density_tile_kernel(StepConst sc, Buffers b, double rho0)
{
    __shared__ __align__(128) float4 srec[kTileCap];
    __shared__ TileRuns g;
    __shared__ __align__(8) uint64_t bar;
    __shared__ double red[4][kTileThreads / 32];
    if (threadIdx.x == 0)
        mbar_init(&bar);
    __syncthreads();
    uint32_t phase = 0;
    const size_t n = sc.n;
    double ea = 0.0, em = 0.0, es = 0.0, ep = 0.0;
    for (uint32_t t = blockIdx.x; t < sc.ntiles; t += gridDim.x) {
        tile_geometry(sc, b.start, t, g);
        if (g.p0 == g.p1)
            continue;
        const bool staged = g.total <= kTileCap;
        if (staged && !stage_tile(g, b.xs32, srec, &bar, phase, b.err))
            return;
        for (uint32_t p = g.p0 + threadIdx.x; p < g.p1; p += blockDim.x) {
            const float4 xi = staged ? srec[g.base[4] + (p - g.slot0[4])] : b.xs32[p];
            float racc = 0.0f;
            for_each_entry(b.nbr, n, p, b.nbr_cnt[p], [&](uint32_t e) {
                const uint32_t r = (e >> kOffBits) / 3, off = e & kOffMask;
                const float4 xj = staged ? srec[g.base[r] + off] : b.xs32[g.slot0[r] + off];
                const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
                const float r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < sc.h2) {
                    const float u = sc.h2 - r2;
                    racc += u * u * u;
                }
            });
            const double d = (double)(sc.mass_poly6 * (sc.h6 + racc)) / rho0 - 1.0;
            ea += fabs(d);
            em = fmax(em, fabs(d));
            es += d;
            ep += d > 0.0 ? d : 0.0;
        }
    }
    ea = warp_sum(ea);
    es = warp_sum(es);
    ep = warp_sum(ep);
    em = warp_max(em);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][w] = ea;
        red[1][w] = em;
        red[2][w] = es;
        red[3][w] = ep;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, m = 0, s = 0, q = 0;
        for (int v = 0; v < kTileThreads / 32; ++v) {
            a += red[0][v];
            m = fmax(m, red[1][v]);
            s += red[2][v];
            q += red[3][v];
        }
        b.partials[4 * (size_t)blockIdx.x + 0] = a;
        b.partials[4 * (size_t)blockIdx.x + 1] = m;
        b.partials[4 * (size_t)blockIdx.x + 2] = s;
        b.partials[4 * (size_t)blockIdx.x + 3] = q;
    }
}

// ------------------------- debug: 16-bit entries -> sorted slot | code << 27

__global__ void __launch_bounds__(kBlock) debug_neighbors_kernel(StepConst sc, Buffers b, uint32_t k)
{
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= sc.n)
        return;
    const size_t n = sc.n;
    uint32_t out = 0xffffffffu;
    if (k < b.nbr_cnt[p]) {
        const int3 c = unpack_cell(b.cell_s[p]);
        const int x0 = (c.x / kTileX) * kTileX, xa = max(x0 - 1, 0);
        const uint32_t e = b.nbr[(size_t)k * n + p];
        const uint32_t code = e >> kOffBits, r = code / 3;
        const int yy = c.y + (int)(r % 3) - 1, zz = c.z + (int)(r / 3) - 1;
        const uint32_t s0 = b.start[((uint32_t)zz * (uint32_t)sc.ny + (uint32_t)yy) * (uint32_t)sc.nx + xa];
        out = (s0 + (e & kOffMask)) | (code << kSlotBits);
    }
    b.dbg_nbr[p] = out;
}

inline unsigned blocks_for(uint32_t n, int bs) { return (unsigned)((n + (uint32_t)bs - 1) / (uint32_t)bs); }

}  // namespace

int tile_grid(int sms) { return sms * occupancy((const void *)lambda_tile_kernel, kTileThreads); }

cudaError_t launch_neighbors(const StepConst &sc, const Buffers &b, cudaStream_t s, int sms, bool)
{
    if (sc.n)
        neighbors_tile_kernel<<<sms * occupancy((const void *)neighbors_tile_kernel, kTileThreads), kTileThreads, 0,
                                s>>>(sc, b);
    return cudaGetLastError();
}

cudaError_t launch_levels(const StepConst &sc, const Buffers &b, cudaStream_t s)
{
    if (!sc.n)
        return cudaGetLastError();
    tile_level_kernel<<<blocks_for(sc.ntiles * 32u, 256), 256, 0, s>>>(sc, b);
    // particles: |P_l| and the neighbour pairs per level
    PartArgs pa{b.lvl_s, b.nbr_cnt, sc.n, sc.n_max, sc.K, sc.part_blocks, b.lvl_hist, b.lvl_off, nullptr,
                b.lvl_count, b.counters + 2};
    part_hist_kernel<<<sc.part_blocks, kPartBlock, 2 * pa.nbins * sizeof(uint32_t), s>>>(pa);
    part_scan_kernel<<<1, 1024, 0, s>>>(pa);
    // tiles: highest level first, empty tiles (level 0) last
    PartArgs ta{b.tile_lvl, nullptr, sc.ntiles, sc.n_max, sc.n_max + 1, sc.tile_blocks, b.tile_hist, b.tile_off,
                b.tile_list, b.tile_count, nullptr};
    part_hist_kernel<<<sc.tile_blocks, kPartBlock, 2 * ta.nbins * sizeof(uint32_t), s>>>(ta);
    part_scan_kernel<<<1, 1024, 0, s>>>(ta);
    part_scatter_kernel<<<sc.tile_blocks, kPartBlock, 32 * ta.nbins * sizeof(uint32_t), s>>>(ta);
    return cudaGetLastError();
}

cudaError_t launch_lambda(const StepConst &sc, const Buffers &b, cudaStream_t s, uint32_t l, int sms)
{
    if (sc.n)
        lambda_tile_kernel<<<sms * occupancy((const void *)lambda_tile_kernel, kTileThreads), kTileThreads, 0, s>>>(
            sc, b, l);
    return cudaGetLastError();
}

cudaError_t launch_deltap(const StepConst &sc, const Buffers &b, cudaStream_t s, uint32_t l, int sms)
{
    if (!sc.n)
        return cudaGetLastError();
    if (sc.scorr_n == 4)
        deltap_tile_kernel<4><<<sms * occupancy((const void *)deltap_tile_kernel<4>, kTileThreads), kTileThreads, 0,
                                s>>>(sc, b, l);
    else
        deltap_tile_kernel<-1><<<sms * occupancy((const void *)deltap_tile_kernel<-1>, kTileThreads), kTileThreads,
                                 0, s>>>(sc, b, l);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const StepConst &sc, const Buffers &b, cudaStream_t s, int sms)
{
    if (sc.n)
        finalize_tile_kernel<<<sms * occupancy((const void *)finalize_tile_kernel, kTileThreads), kTileThreads, 0,
                               s>>>(sc, b);
    return cudaGetLastError();
}

cudaError_t launch_density(const StepConst &sc, const Buffers &b, cudaStream_t s, int sms, int *nblocks)
{
    const int nb = sms * occupancy((const void *)density_tile_kernel, kTileThreads);
    *nblocks = sc.n ? nb : 0;
    if (sc.n)
        density_tile_kernel<<<nb, kTileThreads, 0, s>>>(sc, b, (double)sc.rho0);
    return launch_density_final(sc, b, s, *nblocks);
}

cudaError_t launch_debug_neighbors(const StepConst &sc, const Buffers &b, cudaStream_t s, uint32_t k)
{
    if (sc.n)
        debug_neighbors_kernel<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc, b, k);
    return cudaGetLastError();
}

}  // namespace apbf
