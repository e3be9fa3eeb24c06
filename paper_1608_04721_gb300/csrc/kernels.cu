// CUDA kernels of one Adaptive Position-Based Fluids step (Fig. 7, Sec. 5),
// written for sm_103a. Host orchestration lives in apbf_capi.cu.
//
// Data layout (structure of arrays, sorted by cell after the reorder):
//   state_x, state_v  float4 per particle (w unused), the state between steps
//   recA / recB       16 bytes per particle: position in fixed point (xyz, see
//                     below) and lambda (w, FP32); the two Jacobi buffers
//   xs32              float4 absolute predicted position (FP32), for the
//                     neighbour predicate
//   xt                16 bytes: start-of-step position in fixed point
//   nbr               u32 neighbour entries in blocks of 4 per list column:
//                     entry k of column t at ((k/4)*n + t)*4 + k%4 (a thread
//                     reads a block with one 16-byte load; a warp of
//                     consecutive columns reads 512 contiguous bytes), each
//                     the neighbour's sorted slot. Each list is padded to
//                     whole blocks with entries naming slot n, whose record
//                     (recA, recB and xt hold n + 1) lies far from every
//                     particle, so the solver reads whole blocks without
//                     bounds checks.
//
// Positions inside the solver are 32-bit integers: units of u = 2^e metres
// (2^22 u >= h > 2^21 u, so u <= h / 2^21, 3e-8 m at h = 0.1) relative to the
// scene's grid origin. The difference of two positions is then exact, one
// integer subtraction, at any distance from the origin (a 10 m basin has an
// FP32 spacing of ~1e-6 m). With the bias M = 1.5 * 2^23 added, a difference
// d with |d| < 2^22 is the bit pattern of the float M + d exactly, so one FMA
// (bits as float) * u - M * u gives d * u in metres with no rounding. A larger
// |d| gives a value of magnitude >= 2^22 u >= h, which the kernels treat as
// out of range, as it is; as long as a scene spans fewer than 8e8 units, no
// difference reaches a bit pattern of an infinity or a NaN.
#include "apbf_internal.h"

namespace apbf {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ float3 predict_position(float4 x, float4 v, const StepConst &sc, const DynParams *dyn)
{
    // The prediction step of Fig. 7 in FP32, rounded after every operation (no FMA):
    // v' = v + dt g, x* = x + dt v', then the box clamp.
    float vx = __fadd_rn(v.x, __fmul_rn(sc.dt, sc.g[0]));
    float vy = __fadd_rn(v.y, __fmul_rn(sc.dt, sc.g[1]));
    float vz = __fadd_rn(v.z, __fmul_rn(sc.dt, sc.g[2]));
    float px = __fadd_rn(x.x, __fmul_rn(sc.dt, vx));
    float py = __fadd_rn(x.y, __fmul_rn(sc.dt, vy));
    float pz = __fadd_rn(x.z, __fmul_rn(sc.dt, vz));
    px = fminf(fmaxf(px, dyn->box_lo[0]), dyn->box_hi[0]);
    py = fminf(fmaxf(py, dyn->box_lo[1]), dyn->box_hi[1]);
    pz = fminf(fmaxf(pz, dyn->box_lo[2]), dyn->box_hi[2]);
    return make_float3(px, py, pz);
}

__device__ __forceinline__ int cell_axis(float p, float lo, float inv_h, int dim)
{
    float t = __fmul_rn(__fsub_rn(p, lo), inv_h);
    int c = (int)floorf(t);
    return min(max(c, 0), dim - 1);
}

__device__ __forceinline__ uint32_t pack_cell(int3 c) { return (uint32_t)c.x | ((uint32_t)c.y << 11) | ((uint32_t)c.z << 22); }

__device__ __forceinline__ int3 unpack_cell(uint32_t v)
{
    return make_int3((int)(v & 2047u), (int)((v >> 11) & 2047u), (int)(v >> 22));
}


__device__ __forceinline__ float camera_distance(float4 x, const DynParams *dyn)
{
    float dx = __fsub_rn(x.x, dyn->eye[0]);
    float dy = __fsub_rn(x.y, dyn->eye[1]);
    float dz = __fsub_rn(x.z, dyn->eye[2]);
    float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    d2 = __fadd_rn(d2, __fmul_rn(dz, dz));
    return __fsqrt_rn(d2);
}

// Sec. 4.1 / Eq. 8: linear interpolation of the distance range onto the level
// range, near -> n_max, as K equal-width bins (FP32).
__device__ __forceinline__ uint32_t lod_level(float d, float dmin, float dmax, const StepConst &sc)
{
    float span = __fsub_rn(dmax, dmin);
    float t = 0.0f;
    if (span > 0.0f)
        t = __fdiv_rn(__fsub_rn(d, dmin), span);
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    int b = (int)floorf(__fmul_rn(t, (float)sc.K));
    b = min(b, (int)sc.K - 1);
    return sc.n_max - (uint32_t)b;
}

// Fixed-point solver positions (see the top of this file).
__device__ __forceinline__ long long fx_anchor(float glo, float inv_u)
{
    return __float2ll_rd(__fmul_rn(glo, inv_u));  // the grid origin in units, rounded down
}

// A position in units relative to the anchor: x * 2^-e is exact in FP32, so
// the only rounding is the conversion to the nearest integer.
__device__ __forceinline__ int32_t fx_of(float x, long long anchor, float inv_u)
{
    return (int32_t)(__float2ll_rn(__fmul_rn(x, inv_u)) - anchor);
}

// The FP32 absolute position nearest to a fixed-point one (one rounding).
__device__ __forceinline__ float fx_abs(int32_t a, long long anchor, float u)
{
    return __fmul_rn(__ll2float_rn((long long)a + anchor), u);
}

__device__ __forceinline__ int32_t fx_bits(float v) { return __float_as_int(v); }
__device__ __forceinline__ float fx_word(int32_t v) { return __int_as_float(v); }

// A particle's biased position: (M + x_i / u) mod 2^32, M = kFxMagic.
__device__ __forceinline__ uint32_t fx_biased(float v) { return __float_as_uint(v) + (uint32_t)kFxMagic; }

// The float with the bit pattern (M + (x_i - x_j) / u) mod 2^32 (wrapping, unsigned).
__device__ __forceinline__ float fx_diff_word(uint32_t mi, float vj) { return __uint_as_float(mi - __float_as_uint(vj)); }

// Paired FP32 arithmetic (sm_100 and later): two IEEE round-to-nearest
// operations in one instruction, each lane's result the same bits as the
// scalar operation's.
__device__ __forceinline__ float2 sub2_rn(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rc;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rc, ra, rb;\n\tmov.b64 {%0, %1}, rc;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 mul2_rn(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rc;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rc, ra, rb;\n\tmov.b64 {%0, %1}, rc;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

__device__ __forceinline__ float2 fma2_rn(float2 a, float2 b, float2 c)
{
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}

// Debug-build invariant check (see APBF_DEBUG_CHECKS): true when ok; a failure
// is recorded (the first one's code and index) and the caller keeps its access
// in range. In the release build it is the constant true.
__device__ __forceinline__ bool check_ok(bool ok, uint32_t code, uint32_t index, uint32_t *err, uint32_t *dbg)
{
#if APBF_DEBUG_CHECKS
    if (!ok) {
        atomicOr(err, kErrDebugCheck);
        if (atomicCAS(&dbg[0], 0u, code) == 0u)
            dbg[1] = index;
    }
    return ok;
#else
    (void)code, (void)index, (void)err, (void)dbg;
    return true;
#endif
}

// Programmatic dependent launch: a kernel of the step is launched while its
// predecessor in the stream drains and waits here, before its first global
// memory access, until the predecessor has completed and its writes are
// visible; the launch latency between the step's many short kernels overlaps
// the predecessor's tail.
__device__ __forceinline__ void wait_for_predecessor()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Neighbour batch depth and the minimum resident blocks per SM the solver
// kernels are compiled for (register budget); tuned on the GB300.
#ifndef APBF_LAMBDA_MIN_BLOCKS
#define APBF_LAMBDA_MIN_BLOCKS 5
#endif
#ifndef APBF_DELTAP_MIN_BLOCKS
#define APBF_DELTAP_MIN_BLOCKS 5
#endif
// resident blocks per SM of the deep-batch solver kernels (more registers per thread)
#ifndef APBF_DEEP_MIN_BLOCKS
#define APBF_DEEP_MIN_BLOCKS 3
#endif
constexpr int kUnroll = (int)kEntryBlock;


// Record e of an array through the texture path (see RecTex): the velocity
// pass gathers two records per pair and takes one of them this way, so the two
// gathers are served by the L1's load/store and texture paths side by side.
__device__ __forceinline__ float4 tex_rec(const RecTex &tex, uint32_t e)
{
    const uint4 q = tex1Dfetch<uint4>(tex.t, (int)(e + tex.off));
    return make_float4(__uint_as_float(q.x), __uint_as_float(q.y), __uint_as_float(q.z), __uint_as_float(q.w));
}

// Visit the neighbour entries of one particle in batches of kUnroll: the
// batch's entries are loaded first, then its records, then f runs on each,
// so a thread has kUnroll independent gathers in flight. Entries are read
// once per pass (streaming hint, they should not displace the records that
// neighbouring threads reuse from L1).
// Where the debug-build checks record a failure (unused in the release build).
struct Chk {
    uint32_t *err, *dbg;
};

// DEEP: two entry blocks per batch (2 * kUnroll gathers in flight), for passes
// over so few particles that a thread's chain of dependent loads, not the
// gather throughput, sets the time. A batch's second block past the list is
// all padding (slot n, the far record), whose pairs add exact zeros, so f sees
// the same pairs in the same order and every sum keeps its bits.
template <int UNR = kUnroll, bool DEEP = false, typename F>
__device__ __forceinline__ void for_each_neighbor(const uint32_t *__restrict__ nbr, size_t t, size_t n, uint32_t nn,
                                                  const float4 *__restrict__ rec, Chk chk, F &&f)
{
    static_assert(UNR == (int)kEntryBlock, "one entry block per batch");
    const uint4 *e_ptr = reinterpret_cast<const uint4 *>(nbr) + t;
    if (DEEP) {
        const uint32_t sn = (uint32_t)n;
        const uint4 pad = make_uint4(sn, sn, sn, sn);
        uint4 na = nn ? __ldcs(e_ptr) : pad;
        uint4 nb = nn > (uint32_t)UNR ? __ldcs(e_ptr + n) : pad;
        for (uint32_t k = 0; k < nn; k += 2 * UNR) {
            const uint4 ea = na, eb = nb;
            if (k + 2 * UNR < nn)
                na = __ldcs(e_ptr + (size_t)(k / UNR + 2) * n);
            nb = k + 3 * UNR < nn ? __ldcs(e_ptr + (size_t)(k / UNR + 3) * n) : pad;
            uint32_t e[2 * UNR] = {ea.x, ea.y, ea.z, ea.w, eb.x, eb.y, eb.z, eb.w};
#if APBF_DEBUG_CHECKS
#pragma unroll
            for (int u = 0; u < 2 * UNR; ++u)
                if (!check_ok(e[u] <= n, kCheckNeighbor, (uint32_t)t, chk.err, chk.dbg))
                    e[u] = (uint32_t)n;
#endif
            float4 r[2 * UNR];
#pragma unroll
            for (int u = 0; u < 2 * UNR; ++u)
                r[u] = __ldg(&rec[e[u]]);
#pragma unroll
            for (int u = 0; u < 2 * UNR; ++u)
                f(e[u], r[u]);
        }
        return;
    }
    // the next block's entries are requested before this block's records, so
    // the chain of dependent loads per batch is one load deep, not two
    uint4 nxt = nn ? __ldcs(e_ptr) : make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t k = 0; k < nn; k += UNR) {
        const uint4 eb = nxt;
        if (k + UNR < nn)
            nxt = __ldcs(e_ptr + (size_t)(k / UNR + 1) * n);
        uint32_t e[UNR] = {eb.x, eb.y, eb.z, eb.w};
#if APBF_DEBUG_CHECKS
#pragma unroll
        for (int u = 0; u < UNR; ++u)
            if (!check_ok(e[u] <= n, kCheckNeighbor, (uint32_t)t, chk.err, chk.dbg))
                e[u] = (uint32_t)n;
#endif
        float4 r[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u)
            r[u] = __ldg(&rec[e[u]]);
#pragma unroll
        for (int u = 0; u < UNR; ++u)
            f(e[u], r[u]);
    }
}



template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ float warp_minf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fminf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ float warp_maxf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Block-wide sum of a u32 (any multiple-of-32 block size <= 1024), result in every thread.
__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v, uint32_t *sh32)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0)
        sh32[w] = v;
    __syncthreads();
    uint32_t t = (lane < nw) ? sh32[lane] : 0u;
    t = warp_sum(t);
    return t;
}

// Block-wide exclusive scan of a u32; returns the exclusive prefix, *total the sum.
__device__ __forceinline__ uint32_t block_exclusive_scan_u32(uint32_t v, uint32_t *sh32, uint32_t *total)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o)
            inc += y;
    }
    __syncthreads();
    if (lane == 31)
        sh32[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t s = (lane < nw) ? sh32[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(kFull, s, o);
            if (lane >= o)
                s += y;
        }
        if (lane < nw)
            sh32[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    uint32_t warp_prefix = (w > 0) ? sh32[w - 1] : 0u;
    *total = sh32[nw - 1];
    return warp_prefix + inc - v;
}

// Inclusive scan of one u32 per lane across a warp.
__device__ __forceinline__ uint32_t warp_inclusive_scan_u32(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, v, o);
        if (lane >= o)
            v += y;
    }
    return v;
}

// Single-block scans of E values: warp w of the block owns the contiguous
// segment [w * seg, (w + 1) * seg) (seg a multiple of 32) and walks it in rows
// of 32, so every load and store of a row is one coalesced access.
__device__ __forceinline__ uint32_t warp_segment(uint32_t E)
{
    const uint32_t nw = blockDim.x >> 5;
    return (E + 32u * nw - 1u) / (32u * nw) * 32u;
}

// ------------------------------------------------- per-scene geometry
// A batch concatenates independent scenes; a particle slot's scene is
// constant (cell keys are scene-major, so every order the step uses keeps
// each scene's particles in its own slot range). With one scene (BATCH =
// false) the geometry comes from the kernel constants.

struct Geo {
    float glo[3];
    int nx, ny, nz;
    uint32_t cell_base;
};

template <bool BATCH>
__device__ __forceinline__ uint32_t scene_of(const Buffers &b, uint32_t i)
{
    return BATCH ? (uint32_t)__ldg(&b.sid[i]) : 0u;
}

template <bool BATCH>
__device__ __forceinline__ Geo geo_of(const StepConst &sc, const Buffers &b, uint32_t s)
{
    Geo g;
    if (BATCH) {
        const SceneGeom *t = b.geo + s;
        g.glo[0] = __ldg(&t->glo[0]);
        g.glo[1] = __ldg(&t->glo[1]);
        g.glo[2] = __ldg(&t->glo[2]);
        g.nx = __ldg(&t->nx);
        g.ny = __ldg(&t->ny);
        g.nz = __ldg(&t->nz);
        g.cell_base = __ldg(&t->cell_base);
    } else {
        g.glo[0] = sc.glo[0];
        g.glo[1] = sc.glo[1];
        g.glo[2] = sc.glo[2];
        g.nx = sc.nx;
        g.ny = sc.ny;
        g.nz = sc.nz;
        g.cell_base = 0u;
    }
    return g;
}

__device__ __forceinline__ int3 cell_in(float3 p, const Geo &g, float inv_h)
{
    return make_int3(cell_axis(p.x, g.glo[0], inv_h, g.nx), cell_axis(p.y, g.glo[1], inv_h, g.ny),
                     cell_axis(p.z, g.glo[2], inv_h, g.nz));
}

__device__ __forceinline__ uint32_t key_in(int3 c, const Geo &g)
{
    return g.cell_base + ((uint32_t)c.z * (uint32_t)g.ny + (uint32_t)c.y) * (uint32_t)g.nx + (uint32_t)c.x;
}

// The scene's fixed-point anchors (its grid origin in units).
struct Anchor {
    long long a[3];
};

__device__ __forceinline__ Anchor anchor_of(const Geo &g, const StepConst &sc)
{
    Anchor A;
    for (int k = 0; k < 3; ++k)
        A.a[k] = fx_anchor(g.glo[k], sc.fx_inv_u);
    return A;
}

// ------------------------------------------------------------- a1: range
// The camera-distance range of a step, a pair of words per scene that the
// step's zero fill resets: the minimum as the complement of its bit pattern,
// the maximum as its bit pattern (distances are >= 0, so their patterns order
// like the values, and a zero word stands for "no distance yet" in both).

__device__ __forceinline__ float range_min(const uint32_t *drange, uint32_t s) { return __uint_as_float(~drange[s]); }
__device__ __forceinline__ float range_max(const uint32_t *drange, uint32_t scenes, uint32_t s)
{
    return __uint_as_float(drange[scenes + s]);
}

// Merges each valid thread's distances into its scene's range: one atomic pair
// per block when the block lies in one scene (every block of a single scene).
template <bool BATCH>
__device__ __forceinline__ void range_merge(const StepConst &sc, const Buffers &b, bool valid, uint32_t s, float dmin,
                                            float dmax)
{
    __shared__ float smin[kBlock / 32], smax[kBlock / 32];
    if (!valid) {
        dmin = 3.0e38f;
        dmax = 0.0f;
    }
    const uint32_t s_first = scene_of<BATCH>(b, min(blockIdx.x * blockDim.x, sc.n - 1));
    if (__syncthreads_and(!valid || s == s_first)) {
        dmin = warp_minf(dmin);
        dmax = warp_maxf(dmax);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) {
            smin[w] = dmin;
            smax[w] = dmax;
        }
        __syncthreads();
        if (w == 0) {
            dmin = warp_minf(lane < kBlock / 32 ? smin[lane] : 3.0e38f);
            dmax = warp_maxf(lane < kBlock / 32 ? smax[lane] : 0.0f);
            if (lane == 0 && dmin <= dmax) {
                atomicMax(&b.drange[s_first], ~__float_as_uint(dmin));
                atomicMax(&b.drange[sc.scenes + s_first], __float_as_uint(dmax));
            }
        }
    } else {
        // a block over two or more scenes: one atomic pair per warp and scene
        // (distances are >= 0, so their order is that of their bit patterns)
        const unsigned grp = __match_any_sync(kFull, valid ? s : 0xffffffffu);
        const uint32_t lo = __reduce_max_sync(grp, ~__float_as_uint(dmin));
        const uint32_t hi = __reduce_max_sync(grp, __float_as_uint(dmax));
        if (valid && (threadIdx.x & 31u) == (uint32_t)(__ffs(grp) - 1)) {
            atomicMax(&b.drange[s], lo);
            atomicMax(&b.drange[sc.scenes + s], hi);
        }
    }
}

// ------------------------------------------------- a1: DTVS (Sec. 4.1, Sec. 6)
// Depth image of the particles rendered as spheres, then each particle's
// distance behind the visible surface along its camera ray. Every value that
// decides a level is FP32 with explicit rounding (no contraction): the camera
// basis, the pixel rays, the sphere entry distances, the projection of the
// particle onto its pixel and the distance.

__device__ __forceinline__ float dot3_rn(float a0, float a1, float a2, float b0, float b1, float b2)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(a0, b0), __fmul_rn(a1, b1)), __fmul_rn(a2, b2));
}

__device__ __forceinline__ void normalize3_rn(float &x, float &y, float &z)
{
    const float n = __fsqrt_rn(dot3_rn(x, y, z, x, y, z));
    x = __fdiv_rn(x, n);
    y = __fdiv_rn(y, n);
    z = __fdiv_rn(z, n);
}

// forward f = dir/|dir|, right r = (f x up)/|f x up|, image up u = r x f
struct Basis {
    float f[3], r[3], u[3];
    float ax, ay;  // half extents of the image plane at unit distance
};

__device__ __forceinline__ Basis view_basis(const ViewConst &v, const DynParams *dyn)
{
    Basis B;
    float f0 = dyn->dir[0], f1 = dyn->dir[1], f2 = dyn->dir[2];
    normalize3_rn(f0, f1, f2);
    float r0 = __fsub_rn(__fmul_rn(f1, v.up[2]), __fmul_rn(f2, v.up[1]));
    float r1 = __fsub_rn(__fmul_rn(f2, v.up[0]), __fmul_rn(f0, v.up[2]));
    float r2 = __fsub_rn(__fmul_rn(f0, v.up[1]), __fmul_rn(f1, v.up[0]));
    normalize3_rn(r0, r1, r2);
    B.f[0] = f0;
    B.f[1] = f1;
    B.f[2] = f2;
    B.r[0] = r0;
    B.r[1] = r1;
    B.r[2] = r2;
    B.u[0] = __fsub_rn(__fmul_rn(r1, f2), __fmul_rn(r2, f1));
    B.u[1] = __fsub_rn(__fmul_rn(r2, f0), __fmul_rn(r0, f2));
    B.u[2] = __fsub_rn(__fmul_rn(r0, f1), __fmul_rn(r1, f0));
    B.ax = __fmul_rn(v.tan_half, __fdiv_rn((float)v.W, (float)v.H));
    B.ay = v.tan_half;
    return B;
}

// Image coordinates (pixels, row 0 at the top) of a point relative to the eye
// with depth zc > 0 along f.
__device__ __forceinline__ float2 image_xy(const Basis &B, const ViewConst &v, float q0, float q1, float q2, float zc)
{
    const float qx = __fdiv_rn(__fdiv_rn(dot3_rn(q0, q1, q2, B.r[0], B.r[1], B.r[2]), zc), B.ax);
    const float qy = __fdiv_rn(__fdiv_rn(dot3_rn(q0, q1, q2, B.u[0], B.u[1], B.u[2]), zc), B.ay);
    return make_float2(__fmul_rn(__fadd_rn(qx, 1.0f), __fmul_rn(0.5f, (float)v.W)),
                       __fmul_rn(__fsub_rn(1.0f, qy), __fmul_rn(0.5f, (float)v.H)));
}

// Pixel rays of the current camera; clears the depth image and the binning counters.
__global__ void __launch_bounds__(kBlock) view_rays_kernel(ViewConst v, const DynParams *__restrict__ dyn)
{
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < v.tiles_x * v.tiles_y) {
        v.tile_cnt[p] = 0u;
        v.tile_fill[p] = 0u;
    }
    if (p == 0) {
        *v.big_cnt = 0u;
        *v.list_used = 0ull;
    }
    if (p >= v.W * v.H)
        return;
    const Basis B = view_basis(v, dyn);
    const uint32_t px = p % v.W, py = p / v.W;
    const float sx = __fmul_rn(__fsub_rn(__fdiv_rn((float)(2 * px + 1), (float)v.W), 1.0f), B.ax);
    const float sy = __fmul_rn(__fsub_rn(1.0f, __fdiv_rn((float)(2 * py + 1), (float)v.H)), B.ay);
    float d[3];
    for (int a = 0; a < 3; ++a)
        d[a] = __fadd_rn(__fadd_rn(B.f[a], __fmul_rn(sx, B.r[a])), __fmul_rn(sy, B.u[a]));
    normalize3_rn(d[0], d[1], d[2]);
    v.ray[p] = make_float4(d[0], d[1], d[2], 0.0f);
    v.depth[p] = 0x7f7f7f7fu;
}

// Screen box of a particle's sphere: the pixels around its projection (the
// tangent-plane bounds, or near the camera plane the projections of the 8
// corners of its bounding cube), widened by one pixel (conservative: every
// pixel whose ray enters the sphere is inside). Returns 0 when the sphere is
// not rendered (the eye is inside it) or lies entirely outside the image, 1
// for a box, 2 when a corner is not in front of the camera (then the box is
// the whole image).
struct SplatBox {
    float rel0, rel1, rel2, cc;
    float near;  // a lower bound of every FP32 entry distance into the sphere
    int x0, x1, y0, y1;
};

__device__ __forceinline__ int splat_box(const Basis &B, const ViewConst &v, const DynParams *dyn, float4 x,
                                         SplatBox &o)
{
    o.rel0 = __fsub_rn(x.x, dyn->eye[0]);
    o.rel1 = __fsub_rn(x.y, dyn->eye[1]);
    o.rel2 = __fsub_rn(x.z, dyn->eye[2]);
    const float rad = v.radius, r2 = __fmul_rn(v.radius, v.radius);
    const float len2 = dot3_rn(o.rel0, o.rel1, o.rel2, o.rel0, o.rel1, o.rel2);
    o.cc = __fsub_rn(len2, r2);
    if (!(o.cc > 0.0f))
        return 0;
    // no ray enters the sphere closer than len - r; 4e-6 len (32 units in the
    // last place) covers the rounding of the FP32 entry distance there
    const float len = sqrtf(len2);
    o.near = (len - rad) - 4.0e-6f * len;
    const float zc = dot3_rn(o.rel0, o.rel1, o.rel2, B.f[0], B.f[1], B.f[2]);
    // frustum cull: every pixel ray lies within the angle gamma of f (the image
    // corner), and a ray entering the sphere lies within its angular radius
    // beta of rel, so a sphere whose direction is further than gamma' = gamma +
    // 0.01 rad (rounding) + beta from f is entered by no pixel ray. With
    // cos(beta) = sqrt(cc) / len and sin(beta) = r / len that is
    // zc < sqrt(cc) cos(gamma') - r sin(gamma'). This also drops every sphere
    // behind the camera.
    if (zc < sqrtf(o.cc) * v.cull_cos - rad * v.cull_sin)
        return 0;
    const int W = (int)v.W, H = (int)v.H;
    o.x0 = 0;
    o.x1 = W - 1;
    o.y0 = 0;
    o.y1 = H - 1;
    float fx_lo = 3.0e38f, fx_hi = -3.0e38f, fy_lo = 3.0e38f, fy_hi = -3.0e38f;
    if (zc > 2.0f * rad) {
        // the sphere's exact extent in x/z and y/z: the planes through the
        // eye's vertical (horizontal) axis tangent to the sphere have slopes
        // (c zc +- r sqrt(c^2 + zc^2 - r^2)) / (zc^2 - r^2), c the centre's
        // right (up) coordinate; FP32 rounding moves them by far less than
        // the one-pixel widening below (zc > 2r keeps zc^2 - r^2 well apart)
        const float xc = dot3_rn(o.rel0, o.rel1, o.rel2, B.r[0], B.r[1], B.r[2]);
        const float yc = dot3_rn(o.rel0, o.rel1, o.rel2, B.u[0], B.u[1], B.u[2]);
        const float D = zc * zc - r2, iD = 1.0f / D;
        const float sxq = rad * sqrtf(xc * xc + D), syq = rad * sqrtf(yc * yc + D);
        const float hx = 0.5f * (float)W / B.ax, hy = 0.5f * (float)H / B.ay;
        fx_lo = ((xc * zc - sxq) * iD) * hx + 0.5f * (float)W;
        fx_hi = ((xc * zc + sxq) * iD) * hx + 0.5f * (float)W;
        fy_lo = 0.5f * (float)H - ((yc * zc + syq) * iD) * hy;
        fy_hi = 0.5f * (float)H - ((yc * zc - syq) * iD) * hy;
    } else {
        // near the camera plane: the projections of the 8 corners of the
        // sphere's bounding cube
#pragma unroll 1
        for (int c = 0; c < 8; ++c) {
            const float q0 = __fadd_rn(o.rel0, (c & 1) ? rad : -rad);
            const float q1 = __fadd_rn(o.rel1, (c & 2) ? rad : -rad);
            const float q2 = __fadd_rn(o.rel2, (c & 4) ? rad : -rad);
            const float zq = dot3_rn(q0, q1, q2, B.f[0], B.f[1], B.f[2]);
            if (!(zq > 0.0f))
                return 2;
            const float2 xy = image_xy(B, v, q0, q1, q2, zq);
            fx_lo = fminf(fx_lo, xy.x);
            fx_hi = fmaxf(fx_hi, xy.x);
            fy_lo = fminf(fy_lo, xy.y);
            fy_hi = fmaxf(fy_hi, xy.y);
        }
    }
    if (fx_hi < -1.0f || fy_hi < -1.0f || fx_lo > (float)W + 1.0f || fy_lo > (float)H + 1.0f)
        return 0;
    o.x0 = max((int)floorf(fmaxf(fx_lo, -1.0f)) - 1, 0);
    o.x1 = min((int)floorf(fminf(fx_hi, (float)W + 1.0f)) + 1, W - 1);
    o.y0 = max((int)floorf(fmaxf(fy_lo, -1.0f)) - 1, 0);
    o.y1 = min((int)floorf(fminf(fy_hi, (float)H + 1.0f)) + 1, H - 1);
    return (o.x0 <= o.x1 && o.y0 <= o.y1) ? 1 : 0;
}

// Entry distance of the ray into the sphere at rel (FP32, every operation
// rounded), as float bits; 0x7f7f7f7f when it does not enter in front of the eye.
__device__ __forceinline__ uint32_t entry_bits(float4 ray, float rel0, float rel1, float rel2, float r2)
{
    const float bb = dot3_rn(ray.x, ray.y, ray.z, rel0, rel1, rel2);
    if (!(bb > 0.0f))
        return 0x7f7f7f7fu;
    const float w0 = __fsub_rn(rel0, __fmul_rn(bb, ray.x));
    const float w1 = __fsub_rn(rel1, __fmul_rn(bb, ray.y));
    const float w2 = __fsub_rn(rel2, __fmul_rn(bb, ray.z));
    const float disc = __fsub_rn(r2, dot3_rn(w0, w1, w2, w0, w1, w2));
    if (!(disc >= 0.0f))
        return 0x7f7f7f7fu;
    const float t = __fsub_rn(bb, __fsqrt_rn(disc));
    return t > 0.0f ? __float_as_uint(t) : 0x7f7f7f7fu;
}

// Binning of the spheres into kTilePx x kTilePx pixel tiles, in two phases.
// Phase 0 takes the spheres of particles that had fewer than kFrontNeighbors
// neighbours in the previous step (the fluid's surfaces, which hide most of
// the rest); phase 1 takes the others, after tile_max holds each tile's
// farthest depth of the phase-0 image, and lists a sphere only in the tiles
// where it can still come out in front (its nearest possible entry is
// nearer than that tile's farthest depth: otherwise it can lower no pixel
// of the tile). Pass 0 of a phase reserves room in the tile lists (capacity
// v.list_cap entries) for each sphere's tiles and counts them per tile; a
// sphere that crosses the camera plane, covers more than kMaxSplatTiles
// tiles or finds the lists full is listed as "big" instead. Pass 1 writes
// the tile lists of the spheres pass 0 accepted. Positive floats order like
// their bit patterns, so the depth is a minimum over unsigned integers: it
// depends neither on list order nor on which spheres took which path, and a
// sphere that can lower no pixel may be left out.
// A phase-1 sphere's box as stored in phase 0 when it has none: culled, or
// crossing the camera plane (no real box reaches these codes: x1 < 16384).
constexpr uint32_t kBoxNone = 0xffffffffu, kBoxBig = 0xfffffffeu;

__device__ __forceinline__ bool tile_open(const ViewConst &v, int phase, uint32_t t, float near)
{
    return phase == 0 || near < __uint_as_float(v.tile_max[t]);
}

__global__ void __launch_bounds__(kBlock) splat_bin_kernel(StepConst sc, Buffers b, ViewConst v, int pass, int phase)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < sc.n;
    const bool member = valid && ((b.prev_cnt[i] < kFrontNeighbors) == (phase == 0));
    int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
    float near = 0.0f;
    uint32_t mask = 0;  // pass 0: the open tiles of a box of at most 32 tiles
    if (pass == 1) {
        const bool mine = member && v.accepted[i];
        if (mine) {
            const uint2 bx = v.box[i];
            x0 = (int)(bx.x & 0xffffu);
            x1 = (int)(bx.x >> 16);
            y0 = (int)(bx.y & 0xffffu);
            y1 = (int)(bx.y >> 16);
            near = v.near[i];
        }
        const int tx0 = x0 / kTilePx, tx1 = x1 / kTilePx, ty0 = y0 / kTilePx, ty1 = y1 / kTilePx;
        const int tw = tx1 - tx0 + 1, ntb = mine ? tw * (ty1 - ty0 + 1) : 0;
        // spheres over many tiles: the warp writes their entries together, one
        // tile per lane (each entry's slot comes from an atomic on its tile)
        unsigned wide = __ballot_sync(kFull, ntb > 32);
        const int lane = threadIdx.x & 31;
        while (wide) {
            const int src = __ffs(wide) - 1;
            wide &= wide - 1;
            const int sx0 = __shfl_sync(kFull, tx0, src), sy0 = __shfl_sync(kFull, ty0, src);
            const int sw = __shfl_sync(kFull, tw, src), sn = __shfl_sync(kFull, ntb, src);
            const float snear = __shfl_sync(kFull, near, src);
            const uint32_t si = __shfl_sync(kFull, i, src);
            for (int q = lane; q < sn; q += 32) {
                const uint32_t t = (uint32_t)(sy0 + q / sw) * v.tiles_x + (uint32_t)(sx0 + q % sw);
                if (tile_open(v, phase, t, snear))
                    v.tile_list[v.tile_start[t] + atomicAdd(&v.tile_fill[t], 1u)] = si;
            }
        }
        if (ntb == 0 || ntb > 32)
            return;
        // the tiles recorded open in pass 0: all four atomics of a group are
        // issued before the list writes that wait for them
        uint32_t mk = v.open_mask[i];
        while (mk) {
            uint32_t t4[4], s4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                t4[q] = 0xffffffffu;
                if (mk) {
                    const int bit = __ffs(mk) - 1;
                    mk &= mk - 1u;
                    t4[q] = (uint32_t)(ty0 + bit / tw) * v.tiles_x + (uint32_t)(tx0 + bit % tw);
                    s4[q] = atomicAdd(&v.tile_fill[t4[q]], 1u);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (t4[q] != 0xffffffffu)
                    v.tile_list[v.tile_start[t4[q]] + s4[q]] = i;
        }
        return;
    } else {
        int kind = 0;
        uint32_t nt = 0;
        if (valid)
            v.accepted[i] = 0;
        if (phase == 0 && valid) {
            // every sphere's screen box (it does not depend on the phase): the
            // spheres of phase 1 store theirs here, on lanes that would idle
            // while the few phase-0 spheres are boxed
            const Basis B = view_basis(v, b.dyn);
            SplatBox o;
            kind = splat_box(B, v, b.dyn, b.state_x[i], o);
            if (kind == 1) {
                x0 = o.x0;
                x1 = o.x1;
                y0 = o.y0;
                y1 = o.y1;
                near = o.near;
            }
            if (!member) {
                v.box[i] = kind == 1 ? make_uint2((uint32_t)x0 | ((uint32_t)x1 << 16), (uint32_t)y0 | ((uint32_t)y1 << 16))
                                     : make_uint2(kind == 0 ? kBoxNone : kBoxBig, 0u);
                v.near[i] = near;
            }
        } else if (member) {  // phase 1: the box stored in phase 0
            const uint2 bx = v.box[i];
            kind = bx.x == kBoxNone ? 0 : (bx.x == kBoxBig ? 2 : 1);
            if (kind == 1) {
                x0 = (int)(bx.x & 0xffffu);
                x1 = (int)(bx.x >> 16);
                y0 = (int)(bx.y & 0xffffu);
                y1 = (int)(bx.y >> 16);
                near = v.near[i];
            }
        }
        if (member) {
            if (kind == 1) {
                const int tx0 = x0 / kTilePx, tx1 = x1 / kTilePx, ty0 = y0 / kTilePx, ty1 = y1 / kTilePx;
                if ((uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1)) > kMaxSplatTiles) {
                    kind = 2;
                } else {
                    int bit = 0;
                    for (int ty = ty0; ty <= ty1; ++ty)
                        for (int tx = tx0; tx <= tx1; ++tx, ++bit)
                            if (tile_open(v, phase, (uint32_t)ty * v.tiles_x + (uint32_t)tx, near)) {
                                ++nt;
                                if (bit < 32)
                                    mask |= 1u << bit;
                            }
                    if (nt == 0)
                        kind = 0;  // hidden in every tile it covers
                }
            }
        }
        // one reservation per block: the lanes' tile counts, prefix-summed in
        // each warp, the warps' sums in shared memory (one atomic per warp on
        // the single counter queued up behind each other: 32k per pass)
        __shared__ uint32_t sh_w[kBlock / 32];
        __shared__ unsigned long long sh_base;
        uint32_t incl = nt;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o)
                incl += y;
        }
        if (lane == 31)
            sh_w[w] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t tot = 0;
            for (int k = 0; k < kBlock / 32; ++k) {
                const uint32_t c = sh_w[k];
                sh_w[k] = tot;
                tot += c;
            }
            sh_base = tot ? atomicAdd(v.list_used, (unsigned long long)tot) : 0ull;
        }
        __syncthreads();
        const unsigned long long base = sh_base + sh_w[w];
        if (!member || kind == 0)
            return;
        if (kind == 2 || base + incl > (unsigned long long)v.list_cap) {
            v.big[atomicAdd(v.big_cnt, 1u)] = i;  // whole-image sphere, too many tiles, or the lists are full
            return;
        }
        v.accepted[i] = 1;
        v.box[i] = make_uint2((uint32_t)x0 | ((uint32_t)x1 << 16), (uint32_t)y0 | ((uint32_t)y1 << 16));
        v.near[i] = near;
        v.open_mask[i] = mask;
    }
    // pass 0: count the sphere in each tile it is listed in
    const int tx0 = x0 / kTilePx, tx1 = x1 / kTilePx, ty0 = y0 / kTilePx, ty1 = y1 / kTilePx;
    const int tw = tx1 - tx0 + 1;
    if (tw * (ty1 - ty0 + 1) <= 32) {
        for (uint32_t mk = mask; mk; mk &= mk - 1u) {
            const int bit = __ffs(mk) - 1;
            atomicAdd(&v.tile_cnt[(uint32_t)(ty0 + bit / tw) * v.tiles_x + (uint32_t)(tx0 + bit % tw)], 1u);
        }
        return;
    }
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
            const uint32_t t = (uint32_t)ty * v.tiles_x + (uint32_t)tx;
            if (tile_open(v, phase, t, near))
                atomicAdd(&v.tile_cnt[t], 1u);
        }
}

// Between the phases: each tile's farthest depth of the image so far (an
// empty pixel makes it 3.4e38, so nothing is culled there), and the binning
// counters reset for phase 1.
__global__ void __launch_bounds__(kBlock) splat_tile_max_kernel(ViewConst v)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        *v.big_cnt = 0u;
        *v.list_used = 0ull;
    }
    if (t >= v.tiles_x * v.tiles_y)
        return;
    const uint32_t ox = (t % v.tiles_x) * kTilePx, oy = (t / v.tiles_x) * kTilePx;
    uint32_t m = 0u;
    for (uint32_t y = oy; y < min(oy + kTilePx, v.H); ++y)
        for (uint32_t x = ox; x < min(ox + kTilePx, v.W); ++x)
            m = max(m, v.depth[y * v.W + x]);
    v.tile_max[t] = m;
    v.tile_cnt[t] = 0u;
    v.tile_fill[t] = 0u;
}

// Exclusive scans of the tile counts into tile_start and of the tiles'
// kSplatChunk-entry work chunks into chunk_start (tiles + 1 entries each), one
// block, each warp over a contiguous segment of tiles in coalesced rows.
__global__ void __launch_bounds__(1024) splat_tile_scan_kernel(ViewConst v)
{
    __shared__ uint32_t sh32[32];
    const uint32_t T = v.tiles_x * v.tiles_y;
    const uint32_t seg = warp_segment(T), lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint32_t s0 = min(T, w * seg), s1 = min(T, s0 + seg);
    uint32_t sum = 0, chunks = 0;
    for (uint32_t k = s0 + lane; k < s1; k += 32u) {
        const uint32_t c = v.tile_cnt[k];
        sum += c;
        chunks += (c + kSplatChunk - 1) / kSplatChunk;
    }
    sum = warp_sum(sum);
    chunks = warp_sum(chunks);
    uint32_t total, ctotal;
    uint32_t run = block_exclusive_scan_u32(lane == 0 ? sum : 0u, sh32, &total);
    uint32_t crun = block_exclusive_scan_u32(lane == 0 ? chunks : 0u, sh32, &ctotal);
    run = __shfl_sync(kFull, run, 0);
    crun = __shfl_sync(kFull, crun, 0);
    for (uint32_t r = s0; r < s1; r += 32u) {
        const uint32_t k = r + lane;
        const uint32_t c = k < s1 ? v.tile_cnt[k] : 0u;
        const uint32_t nch = (c + kSplatChunk - 1) / kSplatChunk;
        const uint32_t inc = warp_inclusive_scan_u32(c), cinc = warp_inclusive_scan_u32(nch);
        if (k < s1) {
            const uint32_t cs = crun + cinc - nch;
            v.tile_start[k] = run + inc - c;
            v.chunk_start[k] = cs;
            for (uint32_t q = 0; q < nch; ++q)
                v.chunk_tile[cs + q] = k;
        }
        run += __shfl_sync(kFull, inc, 31);
        crun += __shfl_sync(kFull, cinc, 31);
    }
    if (threadIdx.x == 0) {
        v.tile_start[T] = total;
        v.chunk_start[T] = ctotal;
    }
}

// Spheres covering many tiles (near the eye), crossing the camera plane, or
// left over when the tile lists are full: work items of one sphere and one
// kBigBlockPx x kBigBlockPx block of the image, spread over a persistent
// grid; the block's threads run over the pixels where that image block
// meets the sphere's screen box, keeping the nearest entry with an atomic
// minimum (a plain read first skips pixels that already hold something
// nearer; values only decrease).
__global__ void __launch_bounds__(kBlock) splat_big_kernel(StepConst sc, Buffers b, ViewConst v)
{
    const uint32_t nb = *v.big_cnt;
    const uint32_t mx = (v.W + kBigBlockPx - 1) / kBigBlockPx, my = (v.H + kBigBlockPx - 1) / kBigBlockPx;
    const uint32_t per = mx * my;
    const Basis B = view_basis(v, b.dyn);
    const float r2 = __fmul_rn(v.radius, v.radius);
    for (unsigned long long w = blockIdx.x; w < (unsigned long long)nb * per; w += gridDim.x) {
        const uint32_t k = (uint32_t)(w / per), j = (uint32_t)(w % per);
        const int bx0 = (int)((j % mx) * kBigBlockPx), by0 = (int)((j / mx) * kBigBlockPx);
        SplatBox o;
        if (splat_box(B, v, b.dyn, b.state_x[v.big[k]], o) == 0)
            continue;
        const int x0 = max(o.x0, bx0), x1 = min(o.x1, bx0 + kBigBlockPx - 1);
        const int y0 = max(o.y0, by0), y1 = min(o.y1, by0 + kBigBlockPx - 1);
        if (x0 > x1 || y0 > y1)
            continue;
        const uint32_t bw = (uint32_t)(x1 - x0 + 1), area = bw * (uint32_t)(y1 - y0 + 1);
        for (uint32_t q = threadIdx.x; q < area; q += blockDim.x) {
            const uint32_t p = (uint32_t)(y0 + (int)(q / bw)) * v.W + (uint32_t)(x0 + (int)(q % bw));
            const uint32_t tb = entry_bits(__ldg(&v.ray[p]), o.rel0, o.rel1, o.rel2, r2);
            if (tb < *(volatile uint32_t *)&v.depth[p])
                atomicMin(&v.depth[p], tb);
        }
    }
}

// Persistent blocks over work chunks (up to kSplatChunk list entries of one
// tile): one thread per pixel of the chunk's tile, the spheres staged in
// shared memory kTilePx^2 at a time with their screen boxes, the nearest
// entry along the thread's ray kept in a register (a sphere is tested only
// at pixels inside its conservative box), then merged into the image with an
// atomic minimum (several chunks of a crowded tile may finish in any order).
__global__ void __launch_bounds__(kTilePx *kTilePx) splat_tile_kernel(StepConst sc, Buffers b, ViewConst v)
{
    static_assert(kTilePx == 8, "one bit per pixel of a tile in a 64-bit mask");
    __shared__ float4 sp[kTilePx * kTilePx];
    __shared__ unsigned long long smask[kTilePx * kTilePx];  // pixels of the tile inside each sphere's box
    const uint32_t T = v.tiles_x * v.tiles_y;
    const uint32_t nwork = v.chunk_start[T];
    const float r2 = __fmul_rn(v.radius, v.radius);
    const DynParams *dyn = b.dyn;
    const float e0 = dyn->eye[0], e1 = dyn->eye[1], e2 = dyn->eye[2];
    for (uint32_t w = blockIdx.x; w < nwork; w += gridDim.x) {
        const uint32_t tile = v.chunk_tile[w];  // chunk_start[tile] <= w < chunk_start[tile + 1]
        const uint32_t beg = v.tile_start[tile] + (w - v.chunk_start[tile]) * kSplatChunk;
        const uint32_t end = min(beg + kSplatChunk, v.tile_start[tile + 1]);
        const uint32_t px0 = (tile % v.tiles_x) * kTilePx, py0 = (tile / v.tiles_x) * kTilePx;
        const uint32_t px = px0 + (threadIdx.x % kTilePx);
        const uint32_t py = py0 + (threadIdx.x / kTilePx);
        const bool inside = px < v.W && py < v.H;
        const uint32_t p = py * v.W + px;
        const float4 ray = inside ? v.ray[p] : make_float4(0.0f, 0.0f, 1.0f, 0.0f);
        uint32_t best = 0x7f7f7f7fu;
        for (uint32_t c = beg; c < end; c += kTilePx * kTilePx) {
            const uint32_t k = c + threadIdx.x;
            if (k < end) {
                const uint32_t i = v.tile_list[k];
                const float4 x = b.state_x[i];
                sp[threadIdx.x] = make_float4(__fsub_rn(x.x, e0), __fsub_rn(x.y, e1), __fsub_rn(x.z, e2), 0.0f);
                // the box clipped to the tile as a pixel mask: bit 8 row + column
                const uint2 bx = v.box[i];
                const int c0 = max((int)(bx.x & 0xffffu) - (int)px0, 0), c1 = min((int)(bx.x >> 16) - (int)px0, 7);
                const int r0 = max((int)(bx.y & 0xffffu) - (int)py0, 0), r1 = min((int)(bx.y >> 16) - (int)py0, 7);
                unsigned long long mk = 0ull;
                if (c0 <= c1 && r0 <= r1) {
                    const unsigned long long row = (0xffull >> (7 - (c1 - c0))) << c0;
                    const unsigned long long rows = (r1 == 7 ? ~0ull : ((1ull << (8 * (r1 + 1))) - 1ull)) &
                                                    ~((1ull << (8 * r0)) - 1ull);
                    mk = (row * 0x0101010101010101ull) & rows;
                }
                smask[threadIdx.x] = mk;
            }
            __syncthreads();
            const uint32_t m = min((uint32_t)(kTilePx * kTilePx), end - c);
            if (inside)
                for (uint32_t j = 0; j < m; ++j) {
                    // this warp's 32 pixels (half the tile): skip the sphere together
                    const uint32_t wm = (uint32_t)(smask[j] >> (threadIdx.x & 32u));
                    if (wm == 0u || !((wm >> (threadIdx.x & 31u)) & 1u))
                        continue;
                    const float4 q = sp[j];
                    best = min(best, entry_bits(ray, q.x, q.y, q.z, r2));
                }
            __syncthreads();
        }
        if (inside && best < *(volatile uint32_t *)&v.depth[p])
            atomicMin(&v.depth[p], best);
    }
}

// Distance of each particle behind the visible surface (-1 outside the view)
// and the min/max over the particles in view.
__global__ void __launch_bounds__(kBlock) dtvs_distance_kernel(StepConst sc, Buffers b, ViewConst v)
{
    __shared__ float smin[kBlock / 32], smax[kBlock / 32];
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    float dmin = 3.0e38f, dmax = 0.0f;
    if (i < sc.n) {
        const DynParams *dyn = b.dyn;
        const Basis B = view_basis(v, dyn);
        const float4 x = b.state_x[i];
        const float rel0 = __fsub_rn(x.x, dyn->eye[0]), rel1 = __fsub_rn(x.y, dyn->eye[1]),
                    rel2 = __fsub_rn(x.z, dyn->eye[2]);
        float d = -1.0f;
        const float zc = dot3_rn(rel0, rel1, rel2, B.f[0], B.f[1], B.f[2]);
        if (zc > 0.0f) {
            const float2 xy = image_xy(B, v, rel0, rel1, rel2, zc);
            if (xy.x >= 0.0f && xy.x < (float)v.W && xy.y >= 0.0f && xy.y < (float)v.H) {
                const uint32_t p = (uint32_t)floorf(xy.y) * v.W + (uint32_t)floorf(xy.x);
                const float front = __fsub_rn(__fsqrt_rn(dot3_rn(rel0, rel1, rel2, rel0, rel1, rel2)), v.radius);
                const float g = __fsub_rn(front, __uint_as_float(v.depth[p]));
                d = g > 0.0f ? g : 0.0f;
                dmin = d;
                dmax = d;
            }
        }
        b.lodd[i] = d;
    }
    dmin = warp_minf(dmin);
    dmax = warp_maxf(dmax);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        smin[w] = dmin;
        smax[w] = dmax;
    }
    __syncthreads();
    if (w == 0) {
        dmin = warp_minf(lane < kBlock / 32 ? smin[lane] : 3.0e38f);
        dmax = warp_maxf(lane < kBlock / 32 ? smax[lane] : 0.0f);
        if (lane == 0 && dmin <= dmax) {
            atomicMax(&b.drange[0], ~__float_as_uint(dmin));
            atomicMax(&b.drange[1], __float_as_uint(dmax));
        }
    }
}

// ------------------------------------- a1-a4: range, predict, hash, count
// The prediction and cell hash of every particle, the cell histogram, and
// (distance-to-camera LOD) the camera-distance range of the positions at the
// start of the step; the levels follow from the range in the reorder pass.

template <bool BATCH>
__global__ void __launch_bounds__(kBlock) predict_hash_kernel(StepConst sc, Buffers b, int diag)
{
    wait_for_predecessor();
    const bool range = !diag && sc.lod_mode == APBF_LOD_DTC;
    float dmin = 3.0e38f, dmax = 0.0f;  // this thread's distances (a single scene loops over several)
    bool any = false;
    uint32_t s = 0;
    // block-uniform loop: a batch's grid covers every particle once (one
    // scene per thread); a single scene's grid is capped, which keeps the
    // range's atomics few
    for (uint32_t base = blockIdx.x * blockDim.x; base < sc.n; base += gridDim.x * blockDim.x) {
        const uint32_t i = base + threadIdx.x;
        const bool valid = i < sc.n;
        uint32_t key = 0xffffffffu;
        if (valid) {
            s = scene_of<BATCH>(b, i);
            const Geo g = geo_of<BATCH>(sc, b, s);
            const DynParams *dyn = b.dyn + s;
            float4 x = b.state_x[i];
            float3 p;
            if (diag) {
                p = make_float3(x.x, x.y, x.z);
            } else {
                if (range) {
                    const float d = camera_distance(x, dyn);
                    dmin = fminf(dmin, d);
                    dmax = fmaxf(dmax, d);
                    any = true;
                }
                p = predict_position(x, b.state_v[i], sc, dyn);
            }
            key = key_in(cell_in(p, g, sc.inv_h), g);
            if (!check_ok(key < sc.ncell, kCheckCellKey, i, b.err, b.dbg))
                key = sc.ncell - 1;
            b.key[i] = key;
        }
        // warp-aggregated histogram: one atomic per distinct cell in the warp
        unsigned peers = __match_any_sync(kFull, key);
        int lane = threadIdx.x & 31;
        int leader = __ffs(peers) - 1;
        uint32_t slot0 = 0;
        if (valid && lane == leader)
            slot0 = atomicAdd(&b.cnt[key], (uint32_t)__popc(peers));
        slot0 = __shfl_sync(peers, slot0, leader);
        if (valid)
            b.slot[i] = slot0 + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    }
    if (range)  // uniform over the grid
        range_merge<BATCH>(sc, b, any, s, dmin, dmax);
}

// ------------------------------------------------ a4/a6: scan = cell start

__global__ void __launch_bounds__(1024) scan_reduce_kernel(const uint32_t *__restrict__ cnt, uint32_t ncell,
                                                           uint32_t *__restrict__ tile_sums)
{
    wait_for_predecessor();
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
                                                          uint32_t *__restrict__ start, uint32_t n, Chk chk)
{
    wait_for_predecessor();
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
    if (ncell && base <= ncell - 1 && ncell - 1 < base + 4)  // the last cell: every particle counted
        check_ok(run == n, kCheckScanTotal, run, chk.err, chk.dbg);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        start[ncell] = n;
}

// ------------------------------------------ a4: slot scatter (particle ids)

__global__ void __launch_bounds__(kBlock) scatter_kernel(StepConst sc, Buffers b)
{
    wait_for_predecessor();
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < sc.n)
        b.tmp[b.start[b.key[i]] + b.slot[i]] = b.state_id[i];
}

// ------------------------------------------ a1, a4/a5: level, stable rank + reorder
// Each particle's level (Sec. 4.1, Eq. 8) from the range the predict pass
// reduced (or the camera's range), its sorted slot, and its records in sorted
// order. With an active-set partition the pass also counts the particles of
// each level in each tile of kLevelTile sorted slots (one atomic per distinct
// (level, tile) in a warp; the counts start at zero with the step).

template <bool BATCH>
__global__ void __launch_bounds__(kBlock) reorder_kernel(StepConst sc, Buffers b, int diag)
{
    wait_for_predecessor();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t hist_key = 0xffffffffu;  // bin * level_tiles + tile, or none
    if (i < sc.n) {
        const uint32_t k = b.key[i];
        const uint32_t s0 = b.start[k], s1 = b.start[k + 1];
        // order within a cell by particle id: rank = number of this cell's
        // particles with a smaller id (the slots hold ids in atomic arrival order)
        const uint32_t id = b.state_id[i];
        uint32_t r = 0;
        for (uint32_t j = s0; j < s1; ++j)
            r += (b.tmp[j] < id) ? 1u : 0u;
        const uint32_t p = s0 + r;
        if (check_ok(s1 <= sc.n && p < s1, kCheckSortedSlot, i, b.err, b.dbg)) {
            const uint32_t s = scene_of<BATCH>(b, i);
            const Geo g = geo_of<BATCH>(sc, b, s);
            const DynParams *dyn = b.dyn + s;
            float4 x = b.state_x[i];
            float3 xp = diag ? make_float3(x.x, x.y, x.z) : predict_position(x, b.state_v[i], sc, dyn);
            int3 c = cell_in(xp, g, sc.inv_h);
            b.xs32[p] = make_float4(xp.x, xp.y, xp.z, 0.0f);
            b.cell_s[p] = pack_cell(c);
            if (!diag) {
                const Anchor A = anchor_of(g, sc);
                const float iu = sc.fx_inv_u;
                b.recA[p] = make_float4(fx_word(fx_of(xp.x, A.a[0], iu)), fx_word(fx_of(xp.y, A.a[1], iu)),
                                        fx_word(fx_of(xp.z, A.a[2], iu)), 0.0f);
                b.xt[p] = make_float4(fx_word(fx_of(x.x, A.a[0], iu)), fx_word(fx_of(x.y, A.a[1], iu)),
                                      fx_word(fx_of(x.z, A.a[2], iu)), 0.0f);
                b.id_s[p] = id;
                uint32_t lv = sc.n_max;
                if (sc.lod_mode != APBF_LOD_FIXED) {
                    float dmin = dyn->d_near, dmax = dyn->d_far;
                    if (dyn->auto_range) {
                        dmin = range_min(b.drange, s);
                        dmax = range_max(b.drange, sc.scenes, s);
                    }
                    if (sc.lod_mode == APBF_LOD_DTC) {
                        lv = lod_level(camera_distance(x, dyn), dmin, dmax, sc);
                    } else {  // DTVS: outside the view -> dtvs_outside (n_min unless set)
                        const float d = b.lodd[i];
                        lv = d < 0.0f ? sc.dtvs_outside : lod_level(d, dmin, dmax, sc);
                    }
                }
                b.lvl[i] = (uint8_t)lv;
                b.lvl_s[p] = (uint8_t)lv;
                hist_key = (sc.n_max - lv) * sc.level_tiles + p / kLevelTile;
            }
        }
    }
    if (!diag && sc.lod_mode != APBF_LOD_FIXED && sc.K > 1) {  // the partition's counts (uniform over the grid)
        const unsigned peers = __match_any_sync(kFull, hist_key);
        if (hist_key != 0xffffffffu && (threadIdx.x & 31u) == (uint32_t)(__ffs(peers) - 1))
            atomicAdd(&b.lvl_hist[hist_key], (uint32_t)__popc(peers));
    }
}

// ------------------------------------- neighbour lists (Fig. 7, neighbour search)

// Thread p takes the particle in sorted slot p. With a level partition
// (part), the block is one tile of kLevelTile slots and first places its
// particles in the active list (see level_scan_kernel): particle p goes to
// position t = its bin's offset for the tile + the particles of its bin in
// the tile before it, act[t] = p, and its list is written into column t
// (entry k at k*n + t), so every iteration reads a contiguous prefix of
// columns. Without a partition, column = sorted slot. The entries name
// neighbours by sorted slot either way.
template <bool BATCH>
__global__ void __launch_bounds__(kBlock) neighbors_kernel(StepConst sc, Buffers b, int part)
{
    static_assert(kLevelTile == kBlock, "a block of the neighbour search is one tile of the level partition");
    wait_for_predecessor();
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) {  // the padding entries' record: at least 3h from every particle on every axis
        const float4 far = make_float4(fx_word(kFxFar), fx_word(kFxFar), fx_word(kFxFar), 0.0f);
        b.recA[sc.n] = far;
        b.recB[sc.n] = far;
        b.xt[sc.n] = far;
    }
    uint32_t cnt = 0, bin = 0, t = p;
    if (part) {  // uniform over the grid
        // the stable partition by level: each warp's count per bin, then the
        // particle's rank among its bin in the tile
        extern __shared__ uint32_t wc[];  // (kBlock / 32) warps x K bins
        const uint32_t K = sc.K;
        for (uint32_t k = threadIdx.x; k < (kBlock / 32) * K; k += blockDim.x)
            wc[k] = 0u;
        __syncthreads();
        const bool valid = p < sc.n;
        bin = valid ? sc.n_max - b.lvl_s[p] : 0xffffffffu;
        if (valid && !check_ok(bin < K, kCheckActiveCount, p, b.err, b.dbg))
            bin = K - 1;
        const unsigned peers = __match_any_sync(kFull, bin);
        const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
        if (valid && lane == (uint32_t)(__ffs(peers) - 1))
            wc[w * K + bin] = (uint32_t)__popc(peers);
        __syncthreads();
        if (valid) {
            t = b.lvl_off[(size_t)bin * sc.level_tiles + blockIdx.x] + (uint32_t)__popc(peers & ((1u << lane) - 1u));
            for (uint32_t v = 0; v < w; ++v)
                t += wc[v * K + bin];
            if (!check_ok(t < sc.n, kCheckActiveCount, p, b.err, b.dbg))
                t = p;
            b.act[t] = p;
        } else {
            bin = 0;
        }
    }
    if (p < sc.n) {
        const Geo g = geo_of<BATCH>(sc, b, scene_of<BATCH>(b, p));
        const float4 xi = b.xs32[p];
        const int3 c = unpack_cell(b.cell_s[p]);
        const size_t n = sc.n;
        uint4 *eblk = reinterpret_cast<uint4 *>(b.nbr) + t;  // entry blocks of column t, stride n
        uint4 eb = make_uint4(0u, 0u, 0u, 0u);                // the last four entries written
        // the cells x-1..x+1 of one row (y+dy, z+dz) are contiguous in sorted order
        const int xl = max(c.x - 1, 0), xr = min(c.x + 1, g.nx - 1);
        for (int dz = -1; dz <= 1; ++dz) {
            const int cz = c.z + dz;
            if (cz < 0 || cz >= g.nz)
                continue;
            for (int dy = -1; dy <= 1; ++dy) {
                const int cy = c.y + dy;
                if (cy < 0 || cy >= g.ny)
                    continue;
                const uint32_t row = g.cell_base + ((uint32_t)cz * (uint32_t)g.ny + (uint32_t)cy) * (uint32_t)g.nx;
                const uint32_t j0 = b.start[row + xl], j1 = b.start[row + xr + 1];
                const bool own_row = dy == 0 && dz == 0;  // the only row that holds p itself
                // the window in chunks of up to 32 candidates: first the predicate for each
                // (a hit mask), then one list write per hit, so a warp's lanes share the
                // write loop only as often as the lane with the most hits needs it
                for (uint32_t j = j0; j < j1; j += 32) {
                    const uint32_t je = min(j1, j + 32u);
                    uint32_t hits = 0;
                    for (uint32_t jj = j; jj < je; jj += kUnroll) {
                        float4 xj[kUnroll];
#pragma unroll
                        for (int u = 0; u < kUnroll; ++u)
                            xj[u] = b.xs32[jj + u];  // past je: the next cells (or the slack); masked below
                        uint32_t nib = 0;
#pragma unroll
                        for (int u = 0; u < kUnroll; ++u) {
                            const float2 dxy = sub2_rn(make_float2(xi.x, xi.y), make_float2(xj[u].x, xj[u].y));
                            const float2 sq = mul2_rn(dxy, dxy);
                            const float dz2 = __fsub_rn(xi.z, xj[u].z);
                            float r2 = __fadd_rn(sq.x, sq.y);
                            r2 = __fadd_rn(r2, __fmul_rn(dz2, dz2));
                            if (r2 < sc.h2)
                                nib |= 1u << u;
                        }
                        hits |= nib << (jj - j);
                    }
                    if (je - j < 32u)
                        hits &= (1u << (je - j)) - 1u;
                    if (own_row && p - j < 32u)
                        hits &= ~(1u << (p - j));
                    while (hits) {
                        const uint32_t q = j + (uint32_t)(__ffs(hits) - 1);
                        hits &= hits - 1u;
                        uint32_t qe = q;
#if APBF_DEBUG_CHECKS
                        check_ok(q < sc.n, kCheckNeighbor, t, b.err, b.dbg);
                        if (t == 0 && cnt == 0 && b.dbg[2] != 0u)
                            qe = sc.n + 1u;  // planted: the record past the padding one (inside the arena)
#endif
                        const uint32_t e = qe;
                        eb = make_uint4(eb.y, eb.z, eb.w, e);  // the last four entries, oldest first
                        if (cnt % kEntryBlock == kEntryBlock - 1 && cnt < sc.max_nbr)  // a full block
                            eblk[(size_t)(cnt / kEntryBlock) * n] = eb;
                        ++cnt;
                    }
                }
            }
        }
        if (cnt > sc.max_nbr) {
            atomicOr(b.err, kErrNeighborOverflow);
            atomicOr(&b.err_scene[scene_of<BATCH>(b, p)], kErrNeighborOverflow);
            cnt = sc.max_nbr;
        }
        b.nbr_cnt[t] = (uint8_t)cnt;
        const uint32_t s = cnt % kEntryBlock;
        if (s) {  // the last, partial block, padded
            const uint32_t sentinel = sc.n;
            // its s entries are the last s of eb
            const uint4 out = make_uint4(s == 1 ? eb.w : (s == 2 ? eb.z : eb.y),
                                         s == 1 ? sentinel : (s == 2 ? eb.w : eb.z),
                                         s == 3 ? eb.w : sentinel, sentinel);
            eblk[(size_t)(cnt / kEntryBlock) * n] = out;
        }
    }
    // pair counts: per level bin with a partition (their sum is the total),
    // else the total; one atomic per warp and per distinct bin in it (the
    // counters are few addresses, so atomics from every lane of the warps
    // that straddle a level boundary would queue up behind each other)
    const uint32_t lane = threadIdx.x & 31u;
    if (part) {
        const unsigned grp = __match_any_sync(kFull, bin);
        const uint32_t gsum = __reduce_add_sync(grp, cnt);
        if (lane == (uint32_t)(__ffs(grp) - 1) && gsum)
            atomicAdd(&b.counters[2 + bin], (unsigned long long)gsum);
    } else {
        const uint32_t wsum = warp_sum(cnt);
        if (lane == 0 && wsum)
            atomicAdd(&b.counters[0], (unsigned long long)wsum);
    }
}

// ---------------------------------------- a7: active sets by stable partition
// Particles are partitioned by level, highest first, stable in sorted-slot
// order within a level. P_l is then the prefix of act of length |P_l|.

// The counts per (level bin, tile) come from the reorder pass. Block k of
// this kernel turns bin k's row into exclusive offsets: the particles of the
// bins before it (higher levels) plus those of bin k in the tiles before
// each tile; the offset past the row is |P_l| for l = n_max - k.
__global__ void __launch_bounds__(1024) level_scan_kernel(StepConst sc, Buffers b)
{
    wait_for_predecessor();
    __shared__ uint32_t sh[32];
    // T is a multiple of 4 (level_tile_count), so every row starts on a
    // 16-byte boundary and is read and written four tiles at a time
    const uint32_t T = sc.level_tiles, k = blockIdx.x;
    const uint4 *hist4 = reinterpret_cast<const uint4 *>(b.lvl_hist);
    uint32_t before = 0;
    for (size_t i = threadIdx.x; i < (size_t)k * (T / 4); i += blockDim.x) {
        const uint4 q = hist4[i];
        before += q.x + q.y + q.z + q.w;
    }
    uint32_t carry = block_sum_u32(before, sh);
    const uint4 *row4 = hist4 + (size_t)k * (T / 4);
    uint4 *orow4 = reinterpret_cast<uint4 *>(b.lvl_off) + (size_t)k * (T / 4);
    for (uint32_t c0 = 0; c0 < T / 4; c0 += blockDim.x) {
        const uint32_t c = c0 + threadIdx.x;
        const uint4 v = c < T / 4 ? row4[c] : make_uint4(0u, 0u, 0u, 0u);
        uint32_t total;
        const uint32_t run = carry + block_exclusive_scan_u32(v.x + v.y + v.z + v.w, sh, &total);
        if (c < T / 4)
            orow4[c] = make_uint4(run, run + v.x, run + v.x + v.y, run + v.x + v.y + v.z);
        carry += total;
    }
    if (threadIdx.x == 0) {
        const uint32_t l = sc.n_max - k;  // levels >= l: bins 0..k
        uint32_t c = l <= sc.n_min ? sc.n : carry;
        if (!check_ok(c <= sc.n, kCheckActiveCount, l, b.err, b.dbg))
            c = sc.n;
        b.lvl_count[l] = c;
        if (k == 0) {
            b.lvl_count[sc.n_max + 1] = 0;
            for (uint32_t m = 0; m < sc.n_min; ++m)
                b.lvl_count[m] = sc.n;
        }
    }
}

// ------------------------------------------- contacts with obstacles
// The collision response of Fig. 7 with the obstacles of Sec. 6 (analytic solids): a position
// strictly inside an obstacle moves to the nearest point of its surface.
// Positions are relative to the particle's cell origin og; each obstacle is
// taken relative to og as well, so the arithmetic acts at the scale of the
// obstacle, not of the domain.
__device__ __forceinline__ void project_obstacle(const Obstacle &o, float3 og, float &px, float &py, float &pz)
{
    if (o.kind == APBF_OBSTACLE_SPHERE) {
        const float cx = o.a[0] - og.x, cy = o.a[1] - og.y, cz = o.a[2] - og.z, R = o.b[0];
        const float dx = px - cx, dy = py - cy, dz = pz - cz;
        const float r = sqrtf(dx * dx + dy * dy + dz * dz);
        if (!(r < R))
            return;
        if (r == 0.0f) {
            pz = cz + R;
            return;
        }
        const float k = R / r;
        px = cx + dx * k;
        py = cy + dy * k;
        pz = cz + dz * k;
    } else if (o.kind == APBF_OBSTACLE_BOX) {
        const float lo[3] = {o.a[0] - og.x, o.a[1] - og.y, o.a[2] - og.z};
        const float hi[3] = {o.b[0] - og.x, o.b[1] - og.y, o.b[2] - og.z};
        float p[3] = {px, py, pz};
        float best = 3.0e38f, face = 0.0f;
        int axis = -1;
        for (int k = 0; k < 3; ++k) {
            if (!(p[k] > lo[k] && p[k] < hi[k]))
                return;
            const float dl = p[k] - lo[k], dh = hi[k] - p[k];
            if (dl < best) {
                best = dl;
                axis = k;
                face = lo[k];
            }
            if (dh < best) {
                best = dh;
                axis = k;
                face = hi[k];
            }
        }
        if (axis == 0)
            px = face;
        else if (axis == 1)
            py = face;
        else
            pz = face;
    } else if (o.kind == APBF_OBSTACLE_CONE) {
        const float cx = o.a[0] - og.x, cy = o.a[1] - og.y, cz = o.a[2] - og.z, R = o.b[0], H = o.b[1];
        float ux = px - cx, uy = py - cy;
        const float z = pz - cz;
        const float rho = sqrtf(ux * ux + uy * uy);
        if (!(z > 0.0f && rho / R + z / H < 1.0f))
            return;
        const float L = sqrtf(R * R + H * H);
        const float g = (H * rho + R * z - R * H) / L;  // signed distance to the slant line, < 0 inside
        if (z <= -g) {
            pz = cz;  // the base is nearest
            return;
        }
        const float rho2 = rho - g * H / L, z2 = z - g * R / L;
        if (rho > 0.0f) {
            ux /= rho;
            uy /= rho;
        } else {
            ux = 1.0f;
            uy = 0.0f;
        }
        px = cx + rho2 * ux;
        py = cy + rho2 * uy;
        pz = cz + z2;
    }
}

__device__ __forceinline__ void contact_obstacles(const DynParams *d, float3 og, float &px, float &py, float &pz)
{
    const uint32_t no = d->n_obst;
    for (uint32_t k = 0; k < no; ++k)
        project_obstacle(d->obst[k], og, px, py, pz);
}

// The box in fixed point: the first and last unit inside [box_lo, box_hi].
struct BoxFx {
    int32_t lo[3], hi[3];
};

__device__ __forceinline__ BoxFx box_fx(const DynParams *d, const Anchor &A, float inv_u)
{
    BoxFx k;
    for (int a = 0; a < 3; ++a) {
        k.lo[a] = (int32_t)(__float2ll_ru(__fmul_rn(d->box_lo[a], inv_u)) - A.a[a]);
        k.hi[a] = (int32_t)(__float2ll_rd(__fmul_rn(d->box_hi[a], inv_u)) - A.a[a]);
    }
    return k;
}

// Contacts of a fixed-point position (the collision response of Fig. 7):
// the obstacles in order, then the box. The obstacles act in FP32 relative to
// og, the FP32 position nearest the particle's own: og is a whole number of
// units, so the particle's offset from it and the move back are exact, and the
// arithmetic is at the scale of the obstacle, not of the domain.
__device__ __forceinline__ void obstacles_fx(const DynParams *d, const Anchor &A, const StepConst &sc,
                                             int32_t (&a)[3])
{
    {
        long long ogu[3];
        float og[3], p[3];
        for (int k = 0; k < 3; ++k) {
            og[k] = fx_abs(a[k], A.a[k], sc.fx_u);
            ogu[k] = __float2ll_rn(__fmul_rn(og[k], sc.fx_inv_u));
            p[k] = __fmul_rn(__ll2float_rn((long long)a[k] + A.a[k] - ogu[k]), sc.fx_u);
        }
        contact_obstacles(d, make_float3(og[0], og[1], og[2]), p[0], p[1], p[2]);
        for (int k = 0; k < 3; ++k)
            a[k] = (int32_t)(ogu[k] - A.a[k] + __float2ll_rn(__fmul_rn(p[k], sc.fx_inv_u)));
    }
}

__device__ __forceinline__ void clamp_fx(const BoxFx &bx, int32_t (&a)[3])
{
    for (int k = 0; k < 3; ++k)
        a[k] = min(max(a[k], bx.lo[k]), bx.hi[k]);
}

// The pre-stabilisation loop of Fig. 7 (Sec. 4.3): the particles of level < S are moved out of
// the obstacles and into the box stabil_iters times, the start-of-step
// position (xt) and the prediction (recA) by the same amount, so the
// velocity (x* - x)/dt gains nothing from it.
template <bool BATCH>
__global__ void __launch_bounds__(kBlock) prestab_kernel(StepConst sc, Buffers b)
{
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= sc.n || !(b.lvl_s[p] < sc.stabil_s))
        return;
    const uint32_t s = scene_of<BATCH>(b, p);
    const Geo g = geo_of<BATCH>(sc, b, s);
    const DynParams *d = b.dyn + s;
    const Anchor A = anchor_of(g, sc);
    const BoxFx bx = box_fx(d, A, sc.fx_inv_u);
    const float4 x0f = b.xt[p], xsf = b.recA[p];
    int32_t x0[3] = {fx_bits(x0f.x), fx_bits(x0f.y), fx_bits(x0f.z)};
    int32_t xs[3] = {fx_bits(xsf.x), fx_bits(xsf.y), fx_bits(xsf.z)};
    for (uint32_t it = 0; it < sc.stabil_iters; ++it) {
        int32_t q[3] = {x0[0], x0[1], x0[2]};
        if (d->n_obst)
            obstacles_fx(d, A, sc, q);
        clamp_fx(bx, q);
        for (int k = 0; k < 3; ++k) {
            xs[k] += q[k] - x0[k];
            x0[k] = q[k];
        }
    }
    b.xt[p] = make_float4(fx_word(x0[0]), fx_word(x0[1]), fx_word(x0[2]), x0f.w);
    b.recA[p] = make_float4(fx_word(xs[0]), fx_word(xs[1]), fx_word(xs[2]), xsf.w);
}

// ---------------------------------------------------------- a8: lambda pass

// Eq. 4-6 for one particle: its density over the neighbour list and lambda.
// Every operation is an explicit rounding intrinsic, so that the compiler's
// choice of where to fuse multiply-adds cannot differ between the kernel
// instantiations that inline it (dense or compacted, block size, batch
// depth UNR): a particle's result is the same bits whichever computes it.
template <int UNR = kUnroll, bool DEEP = false>
__device__ __forceinline__ void lambda_one(const StepConst &sc, const float4 *__restrict__ A,
                                           const uint32_t *__restrict__ nbr, size_t t, size_t n, uint32_t nn,
                                           const float4 &ai, Chk chk,
                                           float &lam, float &rho)
{
    float racc = 0.0f, gz = 0.0f, s2 = 0.0f;
    float2 gxy = make_float2(0.0f, 0.0f);
    // the particle's fixed-point position plus the bias: one subtraction per axis
    // gives the bit pattern of M + (x_i - x_j) / u (see the top of this file)
    const uint32_t mx = fx_biased(ai.x), my = fx_biased(ai.y), mz = fx_biased(ai.z);
    const float2 u2 = make_float2(sc.fx_u, sc.fx_u), off2 = make_float2(sc.fx_off, sc.fx_off);
    for_each_neighbor<UNR, DEEP>(nbr, t, n, nn, A, chk, [&](uint32_t e, const float4 &aj) {
        const float2 dxy = fma2_rn(make_float2(fx_diff_word(mx, aj.x), fx_diff_word(my, aj.y)), u2, off2);
        const float dx = dxy.x, dy = dxy.y;
        const float dz = __fmaf_rn(fx_diff_word(mz, aj.z), sc.fx_u, sc.fx_off);
        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
        // branch-free: every pair runs the same instructions; a pair at or past
        // h adds an exact zero (u = 0, gw = 0), and the gradient terms of a
        // coincident pair are exact zeros too (its rsqrt is kept finite by the
        // 1e-30 floor, far below u^2, the smallest nonzero squared distance of
        // the fixed-point positions, and its pair vector is exactly zero), so
        // the sums have the bits of a form that skips those pairs
        const bool in = r2 < sc.h2;
        const float r2c = fminf(r2, sc.h2);
        const float u = __fsub_rn(sc.h2, r2c);
        racc = __fmaf_rn(__fmul_rn(u, u), u, racc);
        const float ir = rsqrtf(fmaxf(r2c, 1.0e-30f));
        const float hr = __fmaf_rn(-r2c, ir, sc.h);
        const float gw = in ? __fmul_rn(__fmul_rn(hr, hr), ir) : 0.0f;
        gxy = fma2_rn(make_float2(gw, gw), dxy, gxy);
        gz = __fmaf_rn(gw, dz, gz);
        s2 = __fmaf_rn(__fmul_rn(gw, gw), r2c, s2);
    });
    rho = __fmul_rn(sc.mass_poly6, __fadd_rn(sc.h6, racc));
    const float C = __fmaf_rn(rho, sc.inv_rho0, -1.0f);
    const float g2 = __fadd_rn(__fmaf_rn(gz, gz, __fmaf_rn(gxy.y, gxy.y, __fmul_rn(gxy.x, gxy.x))), s2);
    const float denom = __fmaf_rn(sc.c_lam, g2, sc.eps);
    lam = __fdiv_rn(-C, denom);
}


// Iteration l, threads over P_{l-1}: particles of P_l compute rho and lambda
// (Eq. 4-6) from A and write (position, lambda) to B; particles that finished
// in iteration l-1 copy their final position into B and keep their lambda
// there, so inactive neighbours enter Eq. 7 with their last lambda.

// Work-list modes of an iteration with a shrinking active set: compacted
// (threads over the level-ordered list act, |P_l| of them) or masked
// (threads over all particles, inactive ones skip). The kernel picks masked
// when |P_l| >= mask_thr * n; the threshold is tuned per scene. Both modes do
// identical arithmetic per particle, so the choice never changes a result.
// In the compacted mode the copies of the particles that finished in
// iteration l-1 (list positions |P_l| .. |P_{l-1}|-1) run as a loop of their
// own, so the loop over P_l is the dense kernel's loop with another bound
// (one loop over P_{l-1} with a branch per particle took 8-10 us more per
// launch on the 1M-particle ocean).
template <bool DENSE, bool DEEP, int BS>
__global__ void __launch_bounds__(BS, (DEEP ? APBF_DEEP_MIN_BLOCKS : APBF_LAMBDA_MIN_BLOCKS) * 256 / BS) lambda_kernel(
    StepConst sc, const float4 *__restrict__ A, float4 *__restrict__ B, float *__restrict__ rho_out,
    const uint32_t *__restrict__ act, const uint32_t *__restrict__ nbr, const uint8_t *__restrict__ nbr_cnt,
    const uint8_t *__restrict__ lvl_s, const uint32_t *__restrict__ lvl_count, uint32_t l, float mask_thr, int part,
    Chk chk)
{
    wait_for_predecessor();
    const size_t n = sc.n;
    const uint32_t t0 = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    // a particle of P_l: rho and lambda (Eq. 4-6) from A, written to B with its position
    auto solve = [&](uint32_t t, uint32_t p) {
        const float4 ai = A[p];
        float lam, rho;
        lambda_one<kUnroll, DEEP>(sc, A, nbr, t, n, nbr_cnt[t], ai, chk, lam, rho);
        B[p] = make_float4(ai.x, ai.y, ai.z, lam);
        rho_out[p] = rho;
    };
    // a particle that finished in iteration l-1: its final position into B, its lambda kept there
    auto keep = [&](uint32_t p) {
        const float4 ai = A[p];
        B[p] = make_float4(ai.x, ai.y, ai.z, B[p].w);
    };
    // grid-stride: at any moment the whole grid works on one compact window of
    // the (cell-sorted) work list, which keeps the gathers' working set in L2;
    // t is the list column (the active-list position with a partition)
    if (DENSE) {
        for (uint32_t t = t0; t < sc.n; t += stride)
            solve(t, part ? act[t] : t);
        return;
    }
    const uint32_t cnt_l = lvl_count[l], cnt_prev = lvl_count[l - 1];
    if ((float)cnt_l >= mask_thr * (float)sc.n) {
        for (uint32_t t = t0; t < sc.n; t += stride) {
            const uint32_t p = part ? act[t] : t;
            const uint32_t lv = lvl_s[p];
            if (lv + 1 < l)
                continue;
            if (lv < l)
                keep(p);
            else
                solve(t, p);
        }
        return;
    }
    for (uint32_t t = cnt_l + t0; t < cnt_prev; t += stride)
        keep(part ? act[t] : t);
    for (uint32_t t = t0; t < cnt_l; t += stride)
        solve(t, part ? act[t] : t);
}

// ------------------------------------------- a9: position correction pass

// x^n for the tensile term (n = 4 unrolled)
template <int NPOW>
__device__ __forceinline__ float powi(float x, uint32_t n)
{
    if (NPOW == 4) {
        const float x2 = __fmul_rn(x, x);
        return __fmul_rn(x2, x2);
    }
    float r = 1.0f;
    for (uint32_t e = 0; e < n; ++e)
        r = __fmul_rn(r, x);
    return r;
}

// The single scene's fixed-point box, read once per kernel (the anchors are
// recomputed where obstacles need them, so they hold no registers in the loop).
struct SceneK {
    BoxFx bx;
    bool obstacles;
};

__device__ __forceinline__ Anchor scene_anchor(const StepConst &sc)
{
    Anchor A;
    for (int a = 0; a < 3; ++a)
        A.a[a] = fx_anchor(sc.glo[a], sc.fx_inv_u);
    return A;
}

__device__ __forceinline__ SceneK scene_k(const StepConst &sc, const DynParams *dyn)
{
    SceneK k;
    k.bx = box_fx(dyn, scene_anchor(sc), sc.fx_inv_u);
    k.obstacles = dyn->n_obst != 0;
    return k;
}

// Eq. 7 for one particle and the contacts after it: the new fixed-point
// position; explicit rounding intrinsics as in lambda_one, so the result does
// not depend on which instantiation computes it.
template <int NPOW, bool BATCH, bool DEEP = false, int UNR = kUnroll>
__device__ __forceinline__ int3 deltap_one(const StepConst &sc, const float4 *__restrict__ B,
                                           const uint32_t *__restrict__ nbr, size_t t, size_t n, uint32_t nn,
                                           const float4 &bi, uint32_t p, const DynParams *__restrict__ dyn,
                                           const Buffers &b, const SceneK &sk)
{
    float2 axy = make_float2(0.0f, 0.0f);
    float az = 0.0f;
    const uint32_t mx = fx_biased(bi.x), my = fx_biased(bi.y), mz = fx_biased(bi.z);
    const float2 u2 = make_float2(sc.fx_u, sc.fx_u), off2 = make_float2(sc.fx_off, sc.fx_off);
    for_each_neighbor<UNR, DEEP>(nbr, t, n, nn, B, Chk{b.err, b.dbg}, [&](uint32_t e, const float4 &bj) {
        const float2 dxy = fma2_rn(make_float2(fx_diff_word(mx, bj.x), fx_diff_word(my, bj.y)), u2, off2);
        const float dx = dxy.x, dy = dxy.y;
        const float dz = __fmaf_rn(fx_diff_word(mz, bj.z), sc.fx_u, sc.fx_off);
        const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
        // as in lambda_one: pairs at or past h and coincident pairs add an exact zero (the
        // tensile term is folded into lambda_i + lambda_j with one FMA)
        const bool in = r2 < sc.h2;
        const float r2c = fminf(fmaxf(r2, 1.0e-30f), sc.h2);
        const float ir = rsqrtf(r2c);
        const float hr = __fmaf_rn(-r2c, ir, sc.h);
        const float gw = in ? __fmul_rn(__fmul_rn(hr, hr), ir) : 0.0f;
        const float u = __fmul_rn(__fsub_rn(sc.h2, r2c), sc.inv_wdq);  // W(r) / W(dq) = u^3
        const float f = __fmul_rn(__fmaf_rn(sc.neg_k, powi<NPOW>(__fmul_rn(__fmul_rn(u, u), u), sc.scorr_n),
                                            __fadd_rn(bi.w, bj.w)), gw);
        axy = fma2_rn(make_float2(f, f), dxy, axy);
        az = __fmaf_rn(f, dz, az);
    });
    // new position in units; contacts: obstacles, then the box
    int32_t a[3] = {fx_bits(bi.x) + __float2int_rn(__fmul_rn(sc.c_dpu, axy.x)),
                    fx_bits(bi.y) + __float2int_rn(__fmul_rn(sc.c_dpu, axy.y)),
                    fx_bits(bi.z) + __float2int_rn(__fmul_rn(sc.c_dpu, az))};
    if (BATCH) {
        // per scene, each bound computed where it is used (fewer live registers)
        const uint32_t s = scene_of<true>(b, p);
        const DynParams *d = dyn + s;
        const SceneGeom *t = b.geo + s;
        if (d->n_obst)
            obstacles_fx(d, anchor_of(geo_of<true>(sc, b, s), sc), sc, a);
        for (int k = 0; k < 3; ++k) {
            const long long ak = fx_anchor(__ldg(&t->glo[k]), sc.fx_inv_u);
            const int32_t lo = (int32_t)(__float2ll_ru(__fmul_rn(d->box_lo[k], sc.fx_inv_u)) - ak);
            const int32_t hi = (int32_t)(__float2ll_rd(__fmul_rn(d->box_hi[k], sc.fx_inv_u)) - ak);
            a[k] = min(max(a[k], lo), hi);
        }
    } else {
        if (sk.obstacles)
            obstacles_fx(dyn, scene_anchor(sc), sc, a);
        clamp_fx(sk.bx, a);
    }
    return make_int3(a[0], a[1], a[2]);
}


// Iteration l, threads over P_l: Eq. 7 with the tensile term from B, box
// contact, Jacobi update written to A.

template <bool DENSE, bool DEEP, int NPOW, bool BATCH, int BS>
__global__ void __launch_bounds__(BS, (DEEP ? APBF_DEEP_MIN_BLOCKS : APBF_DELTAP_MIN_BLOCKS) * 256 / BS) deltap_kernel(
    StepConst sc, const float4 *__restrict__ B, float4 *__restrict__ A, const uint32_t *__restrict__ act,
    const uint32_t *__restrict__ nbr, const uint8_t *__restrict__ nbr_cnt, const uint32_t *__restrict__ cell_s,
    const uint32_t *__restrict__ lvl_count, const DynParams *__restrict__ dyn, Buffers b, uint32_t l, float mask_thr,
    int part)
{
    wait_for_predecessor();
    const uint32_t cnt_l = DENSE ? sc.n : lvl_count[l];
    const bool masked = !DENSE && (float)cnt_l >= mask_thr * (float)sc.n;
    const uint32_t work = masked ? sc.n : cnt_l;
    const size_t n = sc.n;
    const SceneK sk = scene_k(sc, dyn);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < work; t += gridDim.x * blockDim.x) {
        const uint32_t p = part ? act[t] : t;  // t: list column (active-list position with a partition)
        if (masked && b.lvl_s[p] < l)
            continue;
        const float4 bi = B[p];
        const int3 np = deltap_one<NPOW, BATCH, DEEP>(sc, B, nbr, t, n, nbr_cnt[t], bi, p, dyn, b, sk);
        A[p] = make_float4(fx_word(np.x), fx_word(np.y), fx_word(np.z), bi.w);
    }
}

// ------------------------------------------ a10: velocity, XSPH, commit

// Five resident blocks per SM (48 registers instead of 64): the pass waits on
// its two gathers per pair, and the extra warps hide more of that latency
// (1M-particle ocean: 100.4 -> 97.5 us per step; at six blocks it spills).
template <bool BATCH>
__global__ void __launch_bounds__(kBlock, 5) finalize_kernel(StepConst sc, Buffers b, int part)
{
    wait_for_predecessor();
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;  // list column
    if (t == 0) {  // running total of particle-iterations: sum over l >= 1 of |P_l| (Eq. 10)
        unsigned long long it = (unsigned long long)sc.n * sc.n_max;
        if (part) {
            it = 0;
            for (uint32_t l = 1; l <= sc.n_max; ++l)
                it += b.lvl_count[l];
        }
        b.counters[kIterTotalSlot] += it;
    }
    if (t >= sc.n)
        return;
    const uint32_t p = part ? b.act[t] : t;
    const size_t n = sc.n;
    const float4 af = b.recA[p];
    const float4 x0 = b.xt[p];
    // displacement over the step in units (exact), v = displacement * u / dt
    const int32_t dix = fx_bits(af.x) - fx_bits(x0.x), diy = fx_bits(af.y) - fx_bits(x0.y),
                  diz = fx_bits(af.z) - fx_bits(x0.z);
    const float vx = (float)dix * sc.v_scale, vy = (float)diy * sc.v_scale, vz = (float)diz * sc.v_scale;
    const uint32_t mx = fx_biased(af.x), my = fx_biased(af.y), mz = fx_biased(af.z);
    float sx = 0.0f, sy = 0.0f, sz = 0.0f;  // sum of (v_j - v_i) W, velocities in units per step
    const uint32_t nn = b.nbr_cnt[t];
    b.prev_cnt[p] = (uint8_t)nn;  // by state slot, for the next step's depth image
    const uint4 *e_ptr = reinterpret_cast<const uint4 *>(b.nbr) + t;
    uint4 nxt = nn ? __ldcs(e_ptr) : make_uint4(0u, 0u, 0u, 0u);  // next block requested early
    for (uint32_t k = 0; k < nn; k += kUnroll) {
        const uint4 eb = nxt;
        if (k + kUnroll < nn)
            nxt = __ldcs(e_ptr + (size_t)(k / kUnroll + 1) * n);
        uint32_t e[kUnroll] = {eb.x, eb.y, eb.z, eb.w};
#if APBF_DEBUG_CHECKS
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (!check_ok(e[u] <= n, kCheckNeighbor, t, b.err, b.dbg))
                e[u] = (uint32_t)n;
#endif
        float4 aj[kUnroll], xj[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            aj[u] = __ldg(&b.recA[e[u]]);
            xj[u] = b.texXt.t ? tex_rec(b.texXt, e[u]) : __ldg(&b.xt[e[u]]);
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const float dx = fmaf(fx_diff_word(mx, aj[u].x), sc.fx_u, sc.fx_off);
            const float dy = fmaf(fx_diff_word(my, aj[u].y), sc.fx_u, sc.fx_off);
            const float dz = fmaf(fx_diff_word(mz, aj[u].z), sc.fx_u, sc.fx_off);
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < sc.h2) {
                const float w = sc.h2 - r2;
                const float W = w * w * w;
                // (v_j - v_i) in units per step: the difference of the two displacements, exact
                sx += (float)(fx_bits(aj[u].x) - fx_bits(xj[u].x) - dix) * W;
                sy += (float)(fx_bits(aj[u].y) - fx_bits(xj[u].y) - diy) * W;
                sz += (float)(fx_bits(aj[u].z) - fx_bits(xj[u].z) - diz) * W;
            }
        }
    }
    const uint32_t s = scene_of<BATCH>(b, p);
    const Anchor A = anchor_of(geo_of<BATCH>(sc, b, s), sc);
    const DynParams *dyn = b.dyn + s;
    float px = fminf(fmaxf(fx_abs(fx_bits(af.x), A.a[0], sc.fx_u), dyn->box_lo[0]), dyn->box_hi[0]);
    float py = fminf(fmaxf(fx_abs(fx_bits(af.y), A.a[1], sc.fx_u), dyn->box_lo[1]), dyn->box_hi[1]);
    float pz = fminf(fmaxf(fx_abs(fx_bits(af.z), A.a[2], sc.fx_u), dyn->box_lo[2]), dyn->box_hi[2]);
    const float cv = sc.c_xsph * sc.v_scale;
    b.state_x[p] = make_float4(px, py, pz, 0.0f);
    b.state_v[p] = make_float4(vx + cv * sx, vy + cv * sy, vz + cv * sz, 0.0f);
    b.state_id[p] = b.id_s[p];
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

// density diagnostic (Fig. 9): rho at the current positions, FP64 partial sums
__global__ void __launch_bounds__(kBlock) density_kernel(StepConst sc, Buffers b, double rho0)
{
    __shared__ double sh[4][kBlock / 32];
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    double ea = 0.0, em = 0.0, es = 0.0, ep = 0.0;
    if (p < sc.n) {
        const size_t n = sc.n;
        const float4 xi = b.xs32[p];
        float racc = 0.0f;
        const uint32_t nn = b.nbr_cnt[p];
        for (uint32_t k = 0; k < nn; ++k) {
            uint32_t j = b.nbr[entry_index(k, p, n)];
            if (!check_ok(j < sc.n, kCheckNeighbor, p, b.err, b.dbg))
                j = p;
            const float4 xj = b.xs32[j];
            const float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < sc.h2) {
                const float u = sc.h2 - r2;
                racc += u * u * u;
            }
        }
        const double e = (double)(sc.mass_poly6 * (sc.h6 + racc)) / rho0 - 1.0;
        ea = fabs(e);
        em = fabs(e);
        es = e;
        ep = e > 0.0 ? e : 0.0;
    }
    ea = warp_sum(ea);
    es = warp_sum(es);
    ep = warp_sum(ep);
    em = warp_max(em);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][w] = ea;
        sh[1][w] = em;
        sh[2][w] = es;
        sh[3][w] = ep;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, m = 0, s = 0, q = 0;
        for (int v = 0; v < kBlock / 32; ++v) {
            a += sh[0][v];
            m = fmax(m, sh[1][v]);
            s += sh[2][v];
            q += sh[3][v];
        }
        b.partials[4 * (size_t)blockIdx.x + 0] = a;
        b.partials[4 * (size_t)blockIdx.x + 1] = m;
        b.partials[4 * (size_t)blockIdx.x + 2] = s;
        b.partials[4 * (size_t)blockIdx.x + 3] = q;
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

template <bool BATCH>
__global__ void __launch_bounds__(kBlock) debug_xstar_kernel(StepConst sc, Buffers b, const float4 *__restrict__ rec)
{
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= sc.n)
        return;
    const float4 r = rec[p];
    const Anchor A = anchor_of(geo_of<BATCH>(sc, b, scene_of<BATCH>(b, p)), sc);
    b.dbg4[p] = make_float4(fx_abs(fx_bits(r.x), A.a[0], sc.fx_u), fx_abs(fx_bits(r.y), A.a[1], sc.fx_u),
                            fx_abs(fx_bits(r.z), A.a[2], sc.fx_u), 0.0f);
}

__global__ void __launch_bounds__(kBlock) debug_lambda_kernel(StepConst sc, Buffers b, const float4 *__restrict__ rec)
{
    uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < sc.n)
        b.stage_f[p] = rec[p].w;
}

inline unsigned blocks_for(uint32_t n, int bs) { return (unsigned)((n + (uint32_t)bs - 1) / (uint32_t)bs); }

// Resident blocks of kBlock threads per SM for a kernel (cached per function).
int occupancy(const void *fn, int block = kBlock)
{
    static const void *keys[64];
    static int vals[64];
    for (int k = 0; k < 64; ++k)
        if (keys[k] == fn)
            return vals[k];
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, 0) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 4;
    }
    for (int k = 0; k < 64; ++k)
        if (!keys[k]) {
            keys[k] = fn;
            vals[k] = occ;
            break;
        }
    return occ;
}

}  // namespace

// ------------------------------------------------------------- launchers

// Launches k with the programmatic-dependent-launch attribute (see
// wait_for_predecessor); in a captured graph this becomes a programmatic edge.
template <typename... KArgs, typename... Args>
cudaError_t launch_after_smem(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}
template <typename... KArgs, typename... Args>
cudaError_t launch_after(void (*k)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, Args... args)
{
    return launch_after_smem(k, grid, block, 0, s, args...);
}

cudaError_t launch_predict_hash(const StepConst &sc, const Buffers &b, cudaStream_t s, bool diag)
{
    if (sc.n)
        return sc.scenes > 1
                   ? launch_after(predict_hash_kernel<true>, blocks_for(sc.n, kBlock), kBlock, s, sc, b, diag ? 1 : 0)
                   : launch_after(predict_hash_kernel<false>, min(blocks_for(sc.n, kBlock), kPredictBlocks), kBlock, s,
                                  sc, b, diag ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_scan(const StepConst &sc, const Buffers &b, cudaStream_t s)
{
    unsigned tiles = blocks_for(sc.ncell, kScanTile);
    cudaError_t e = launch_after(scan_reduce_kernel, tiles, 1024, s, b.cnt, sc.ncell, b.tile_sums);
    if (e != cudaSuccess)
        return e;
    return launch_after(scan_apply_kernel, tiles, 1024, s, b.cnt, sc.ncell, b.tile_sums, b.start, sc.n,
                        Chk{b.err, b.dbg});
}

cudaError_t launch_scatter(const StepConst &sc, const Buffers &b, cudaStream_t s)
{
    if (sc.n)
        return launch_after(scatter_kernel, blocks_for(sc.n, kBlock), kBlock, s, sc, b);
    return cudaGetLastError();
}

cudaError_t launch_reorder(const StepConst &sc, const Buffers &b, cudaStream_t s, bool diag)
{
    if (sc.n)
        return launch_after(sc.scenes > 1 ? reorder_kernel<true> : reorder_kernel<false>, blocks_for(sc.n, kBlock),
                            kBlock, s, sc, b, diag ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_neighbors(const StepConst &sc, const Buffers &b, cudaStream_t s, bool part)
{
    if (sc.n)
        return launch_after_smem(sc.scenes > 1 ? neighbors_kernel<true> : neighbors_kernel<false>,
                                 blocks_for(sc.n, kBlock), kBlock, part ? (kBlock / 32) * sc.K * sizeof(uint32_t) : 0,
                                 s, sc, b, part ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_levels(const StepConst &sc, const Buffers &b, cudaStream_t s)
{
    if (!sc.n)
        return cudaGetLastError();
    return launch_after(level_scan_kernel, sc.K, 1024, s, sc, b);
}

// The deep-batch solver kernels run every pass of a scene (or batch) with no more
// particles than the regular kernel holds resident threads: there each thread has
// one particle, and its chain of dependent loads, not the gather throughput, sets
// the pass's time (131k-particle dam break 0.294 -> 0.282 ms/step; at 225k
// particles, 1.16 per resident thread, the deep kernels lost 1.3 %). Both
// variants give the same bits.
bool deep_pass(const StepConst &sc, const void *regular, int block, int sms)
{
    return (size_t)sc.n <= (size_t)sms * (size_t)occupancy(regular, block) * (size_t)block;
}

template <int BS>
cudaError_t launch_lambda_bs(const StepConst &sc, const Buffers &b, cudaStream_t s, uint32_t l, bool dense, int sms,
                             float thr)
{
    const int part = partitioned(sc) ? 1 : 0;
    const bool deep = deep_pass(sc, (const void *)lambda_kernel<true, false, BS>, BS, sms);
    auto k = dense ? (deep ? lambda_kernel<true, true, BS> : lambda_kernel<true, false, BS>)
                   : (deep ? lambda_kernel<false, true, BS> : lambda_kernel<false, false, BS>);
    return launch_after(k, sms * occupancy((const void *)k, BS), BS, s, sc, b.recA, b.recB, b.rho, b.act, b.nbr,
                        b.nbr_cnt, b.lvl_s, b.lvl_count, l, thr, part, Chk{b.err, b.dbg});
}

cudaError_t launch_lambda(const StepConst &sc, const Buffers &b, cudaStream_t s, uint32_t l, bool dense, int sms,
                          const Tune &tune)
{
    if (!sc.n)
        return cudaGetLastError();
    return tune.block == 128 ? launch_lambda_bs<128>(sc, b, s, l, dense, sms, tune.mask_threshold)
                             : launch_lambda_bs<256>(sc, b, s, l, dense, sms, tune.mask_threshold);
}

template <bool DENSE, int NPOW, bool BATCH, int BS>
cudaError_t launch_deltap_t(const StepConst &sc, const Buffers &b, cudaStream_t s, uint32_t l, int sms, float thr)
{
    if (deep_pass(sc, (const void *)deltap_kernel<true, false, NPOW, BATCH, BS>, BS, sms)) {
        const int grid = sms * occupancy((const void *)deltap_kernel<DENSE, true, NPOW, BATCH, BS>, BS);
        return launch_after(deltap_kernel<DENSE, true, NPOW, BATCH, BS>, grid, BS, s, sc, b.recB, b.recA, b.act,
                            b.nbr, b.nbr_cnt, b.cell_s, b.lvl_count, b.dyn, b, l, thr, partitioned(sc) ? 1 : 0);
    }
    const int grid = sms * occupancy((const void *)deltap_kernel<DENSE, false, NPOW, BATCH, BS>, BS);
    return launch_after(deltap_kernel<DENSE, false, NPOW, BATCH, BS>, grid, BS, s, sc, b.recB, b.recA, b.act, b.nbr,
                        b.nbr_cnt, b.cell_s, b.lvl_count, b.dyn, b, l, thr, partitioned(sc) ? 1 : 0);
}

template <int BS>
cudaError_t launch_deltap_bs(const StepConst &sc, const Buffers &b, cudaStream_t s, uint32_t l, bool dense, int sms,
                             float thr)
{
    const bool p4 = sc.scorr_n == 4, batch = sc.scenes > 1;
    const int k = (dense ? 4 : 0) + (p4 ? 2 : 0) + (batch ? 1 : 0);
    switch (k) {
    case 0: return launch_deltap_t<false, -1, false, BS>(sc, b, s, l, sms, thr);
    case 1: return launch_deltap_t<false, -1, true, BS>(sc, b, s, l, sms, thr);
    case 2: return launch_deltap_t<false, 4, false, BS>(sc, b, s, l, sms, thr);
    case 3: return launch_deltap_t<false, 4, true, BS>(sc, b, s, l, sms, thr);
    case 4: return launch_deltap_t<true, -1, false, BS>(sc, b, s, l, sms, thr);
    case 5: return launch_deltap_t<true, -1, true, BS>(sc, b, s, l, sms, thr);
    case 6: return launch_deltap_t<true, 4, false, BS>(sc, b, s, l, sms, thr);
    default: return launch_deltap_t<true, 4, true, BS>(sc, b, s, l, sms, thr);
    }
}

cudaError_t launch_deltap(const StepConst &sc, const Buffers &b, cudaStream_t s, uint32_t l, bool dense, int sms,
                          const Tune &tune)
{
    if (!sc.n)
        return cudaGetLastError();
    return tune.block == 128 ? launch_deltap_bs<128>(sc, b, s, l, dense, sms, tune.mask_threshold)
                             : launch_deltap_bs<256>(sc, b, s, l, dense, sms, tune.mask_threshold);
}

cudaError_t launch_finalize(const StepConst &sc, const Buffers &b, cudaStream_t s)
{
    if (!sc.n)
        return cudaGetLastError();
    return launch_after(sc.scenes > 1 ? finalize_kernel<true> : finalize_kernel<false>, blocks_for(sc.n, kBlock),
                        kBlock, s, sc, b, partitioned(sc) ? 1 : 0);
}

cudaError_t launch_prestab(const StepConst &sc, const Buffers &b, cudaStream_t s)
{
    if (sc.n)
        (sc.scenes > 1 ? prestab_kernel<true> : prestab_kernel<false>)<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc,
                                                                                                                    b);
    return cudaGetLastError();
}

cudaError_t launch_dtvs(const StepConst &sc, const Buffers &b, const ViewConst &v, int sms, cudaStream_t s)
{
    const uint32_t pix = v.W * v.H, tiles = v.tiles_x * v.tiles_y;
    view_rays_kernel<<<blocks_for(pix > tiles ? pix : tiles, kBlock), kBlock, 0, s>>>(v, b.dyn);
    if (sc.n) {
        for (int phase = 0; phase < 2; ++phase) {
            if (phase == 1)
                splat_tile_max_kernel<<<blocks_for(tiles, kBlock), kBlock, 0, s>>>(v);
            splat_bin_kernel<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc, b, v, 0, phase);
            splat_tile_scan_kernel<<<1, 1024, 0, s>>>(v);
            splat_bin_kernel<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc, b, v, 1, phase);
            splat_big_kernel<<<(unsigned)(sms > 0 ? 4 * sms : 1), kBlock, 0, s>>>(sc, b, v);
            splat_tile_kernel<<<(unsigned)(sms > 0 ? 32 * sms : 1), kTilePx * kTilePx, 0, s>>>(sc, b, v);
        }
        dtvs_distance_kernel<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc, b, v);
    }
    return cudaGetLastError();
}

cudaError_t launch_unpermute(const StepConst &sc, const Buffers &b, cudaStream_t s, uint32_t what)
{
    if (sc.n)
        unpermute_kernel<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc, b, what);
    return cudaGetLastError();
}

cudaError_t launch_density(const StepConst &sc, const Buffers &b, cudaStream_t s, int *nblocks)
{
    int nb = (int)blocks_for(sc.n, kBlock);
    *nblocks = nb;
    if (sc.n)
        density_kernel<<<nb, kBlock, 0, s>>>(sc, b, (double)sc.rho0);
    density_final_kernel<<<1, 32, 0, s>>>(b.partials, nb, sc.n, b.dstats);
    return cudaGetLastError();
}

cudaError_t launch_debug_xstar(const StepConst &sc, const Buffers &b, const float4 *rec, cudaStream_t s)
{
    if (sc.n)
        (sc.scenes > 1 ? debug_xstar_kernel<true> : debug_xstar_kernel<false>)<<<blocks_for(sc.n, kBlock), kBlock, 0,
                                                                                 s>>>(sc, b, rec);
    return cudaGetLastError();
}

cudaError_t launch_debug_lambda(const StepConst &sc, const Buffers &b, const float4 *rec, cudaStream_t s)
{
    if (sc.n)
        debug_lambda_kernel<<<blocks_for(sc.n, kBlock), kBlock, 0, s>>>(sc, b, rec);
    return cudaGetLastError();
}

int iteration_grid(int sms) { return sms; }

}  // namespace apbf
