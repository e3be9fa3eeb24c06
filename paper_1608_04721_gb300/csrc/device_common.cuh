// Device helpers shared by the CUDA translation units of the APBF step.
#pragma once

#include "apbf_internal.h"

namespace apbf {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ float3 predict_position(float4 x, float4 v, const StepConst &sc, const DynParams *dyn)
{
    // Fig. 7 lines 1-4 in FP32, rounded after every operation (no FMA):
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

__device__ __forceinline__ int3 cell_of(float3 p, const StepConst &sc)
{
    return make_int3(cell_axis(p.x, sc.glo[0], sc.inv_h, sc.nx), cell_axis(p.y, sc.glo[1], sc.inv_h, sc.ny),
                     cell_axis(p.z, sc.glo[2], sc.inv_h, sc.nz));
}

__device__ __forceinline__ uint32_t pack_cell(int3 c) { return (uint32_t)c.x | ((uint32_t)c.y << 11) | ((uint32_t)c.z << 22); }

__device__ __forceinline__ int3 unpack_cell(uint32_t v)
{
    return make_int3((int)(v & 2047u), (int)((v >> 11) & 2047u), (int)(v >> 22));
}

__device__ __forceinline__ float3 cell_origin(int3 c, const StepConst &sc)
{
    return make_float3((float)(sc.m[0] + c.x) * sc.q, (float)(sc.m[1] + c.y) * sc.q, (float)(sc.m[2] + c.z) * sc.q);
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

// Cell-origin difference o_i - o_j = -(offset) q for the 27 neighbour cells.
__device__ __forceinline__ void fill_dtab(float4 *dtab, float q)
{
    if (threadIdx.x < 27) {
        int c = threadIdx.x;
        float ox = (float)(c % 3 - 1), oy = (float)((c / 3) % 3 - 1), oz = (float)(c / 9 - 1);
        dtab[c] = make_float4(-ox * q, -oy * q, -oz * q, 0.0f);
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

}  // namespace apbf
