// apbf_density_stats_static: the density diagnostic of apbf_density_stats for
// caller-provided device positions, with no device allocation at all.
//
// Who needs this: code that may not allocate GPU memory while it runs, for
// example a game or renderer frame loop that forbids cudaMalloc/cudaFree
// mid-frame (they synchronise the device and stall the frame), plugins that
// live inside a host application's fixed memory budget, or callers that
// cannot hand the library an allocator. Every byte of scratch this call needs
// (cell counts, cell starts, slots, the cell-sorted copy of the positions and
// the partial sums) lives in one file-scope __device__ array below, which
// every GPU that loads the library holds until the process exits.
#include <cmath>
#include <mutex>
#include <string>

#include "apbf_internal.h"

namespace apbf {
void set_last_error_message(const std::string &m);
}

namespace {

constexpr uint32_t kMaxParticles = APBF_STATIC_MAX_PARTICLES;
constexpr uint32_t kMaxCells = APBF_STATIC_MAX_CELLS;
constexpr int kSB = 256;
constexpr uint32_t kMaxBlocks = (kMaxParticles + kSB - 1) / kSB;

// Scratch layout in 32-bit words; every region starts on a 16-byte boundary.
constexpr size_t kCount = 0;
constexpr size_t kStart = kCount + kMaxCells;
constexpr size_t kKey = kStart + kMaxCells + 4;
constexpr size_t kSlot = kKey + kMaxParticles;
constexpr size_t kTmp = kSlot + kMaxParticles;
constexpr size_t kSorted = kTmp + kMaxParticles;          // float4 per particle
constexpr size_t kPartial = kSorted + 4 * (size_t)kMaxParticles;  // 4 doubles per block
constexpr size_t kWords = kPartial + 8 * (size_t)kMaxBlocks;

static __device__ __align__(256) uint32_t g_density_scratch[kWords];

std::mutex g_setup_mu;
uint32_t *g_scratch_ptr[64] = {};

struct Params {
    uint32_t n, ncell;
    int nx, ny, nz;
    float glo[3];
    float inv_h, h2, mass_poly6, h6;
    double rho0;
};

__device__ __forceinline__ int axis_cell(float p, float lo, float inv_h, int dim)
{
    const int c = (int)floorf(__fmul_rn(__fsub_rn(p, lo), inv_h));
    return min(max(c, 0), dim - 1);
}

__global__ void hash_count_kernel(Params P, const float *__restrict__ pos, uint32_t *sw)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n)
        return;
    const int cx = axis_cell(pos[3 * i + 0], P.glo[0], P.inv_h, P.nx);
    const int cy = axis_cell(pos[3 * i + 1], P.glo[1], P.inv_h, P.ny);
    const int cz = axis_cell(pos[3 * i + 2], P.glo[2], P.inv_h, P.nz);
    const uint32_t key = ((uint32_t)cz * (uint32_t)P.ny + (uint32_t)cy) * (uint32_t)P.nx + (uint32_t)cx;
    sw[kKey + i] = key;
    sw[kSlot + i] = atomicAdd(&sw[kCount + key], 1u);
}

// one block: exclusive scan of the cell counts into the cell starts
__global__ void __launch_bounds__(1024) start_scan_kernel(Params P, uint32_t *sw)
{
    __shared__ uint32_t warp_tot[32];
    const uint32_t per = (P.ncell + blockDim.x - 1) / blockDim.x;
    const uint32_t c0 = min(P.ncell, threadIdx.x * per), c1 = min(P.ncell, c0 + per);
    uint32_t s = 0;
    for (uint32_t c = c0; c < c1; ++c)
        s += sw[kCount + c];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += y;
    }
    if (lane == 31)
        warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t t = warp_tot[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o)
                t += y;
        }
        warp_tot[lane] = t;
    }
    __syncthreads();
    uint32_t run = (w > 0 ? warp_tot[w - 1] : 0u) + inc - s;
    for (uint32_t c = c0; c < c1; ++c) {
        sw[kStart + c] = run;
        run += sw[kCount + c];
    }
    if (threadIdx.x == 0)
        sw[kStart + P.ncell] = P.n;
}

__global__ void scatter_index_kernel(Params P, uint32_t *sw)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < P.n)
        sw[kTmp + sw[kStart + sw[kKey + i]] + sw[kSlot + i]] = i;
}

// cell-sorted copy of the positions, ties by input index
__global__ void rank_copy_kernel(Params P, const float *__restrict__ pos, uint32_t *sw)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n)
        return;
    const uint32_t k = sw[kKey + i], s0 = sw[kStart + k], s1 = sw[kStart + k + 1];
    uint32_t r = 0;
    for (uint32_t j = s0; j < s1; ++j)
        r += sw[kTmp + j] < i ? 1u : 0u;
    float4 *sorted = reinterpret_cast<float4 *>(sw + kSorted);
    sorted[s0 + r] = make_float4(pos[3 * i + 0], pos[3 * i + 1], pos[3 * i + 2], 0.0f);
}

// rho of every particle over the 27 neighbour cells: pairs are selected by
// the library's FP32 neighbour predicate and summed in its order (row
// windows x-1..x+1 for dz, dy = -1..1, ascending slot), then FP64 partials
__global__ void __launch_bounds__(kSB) density_scan_kernel(Params P, uint32_t *sw)
{
    __shared__ double red[4][kSB / 32];
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    const float4 *sorted = reinterpret_cast<const float4 *>(sw + kSorted);
    double ea = 0.0, em = 0.0, es = 0.0, ep = 0.0;
    if (p < P.n) {
        const float4 xi = sorted[p];
        const int cx = axis_cell(xi.x, P.glo[0], P.inv_h, P.nx);
        const int cy = axis_cell(xi.y, P.glo[1], P.inv_h, P.ny);
        const int cz = axis_cell(xi.z, P.glo[2], P.inv_h, P.nz);
        const int xl = max(cx - 1, 0), xr = min(cx + 1, P.nx - 1);
        float racc = 0.0f;
        for (int dz = -1; dz <= 1; ++dz) {
            const int zz = cz + dz;
            if (zz < 0 || zz >= P.nz)
                continue;
            for (int dy = -1; dy <= 1; ++dy) {
                const int yy = cy + dy;
                if (yy < 0 || yy >= P.ny)
                    continue;
                const uint32_t row = ((uint32_t)zz * (uint32_t)P.ny + (uint32_t)yy) * (uint32_t)P.nx;
                const uint32_t j0 = sw[kStart + row + xl], j1 = sw[kStart + row + xr + 1];
                for (uint32_t j = j0; j < j1; ++j) {
                    if (j == p)
                        continue;
                    const float4 xj = sorted[j];
                    const float ex = __fsub_rn(xi.x, xj.x), ey = __fsub_rn(xi.y, xj.y), ez = __fsub_rn(xi.z, xj.z);
                    float q2 = __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey));
                    q2 = __fadd_rn(q2, __fmul_rn(ez, ez));
                    if (!(q2 < P.h2))
                        continue;
                    const float dx = xi.x - xj.x, dy2 = xi.y - xj.y, dz2 = xi.z - xj.z;
                    const float r2 = dx * dx + dy2 * dy2 + dz2 * dz2;
                    if (r2 < P.h2) {
                        const float u = P.h2 - r2;
                        racc += u * u * u;
                    }
                }
            }
        }
        const double e = (double)(P.mass_poly6 * (P.h6 + racc)) / P.rho0 - 1.0;
        ea = fabs(e);
        em = fabs(e);
        es = e;
        ep = e > 0.0 ? e : 0.0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ea += __shfl_xor_sync(0xffffffffu, ea, o);
        es += __shfl_xor_sync(0xffffffffu, es, o);
        ep += __shfl_xor_sync(0xffffffffu, ep, o);
        em = fmax(em, __shfl_xor_sync(0xffffffffu, em, o));
    }
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
        for (int v = 0; v < kSB / 32; ++v) {
            a += red[0][v];
            m = fmax(m, red[1][v]);
            s += red[2][v];
            q += red[3][v];
        }
        double *part = reinterpret_cast<double *>(sw + kPartial);
        part[4 * blockIdx.x + 0] = a;
        part[4 * blockIdx.x + 1] = m;
        part[4 * blockIdx.x + 2] = s;
        part[4 * blockIdx.x + 3] = q;
    }
}

__global__ void __launch_bounds__(32) stats_final_kernel(Params P, uint32_t *sw, int nblocks, double *out)
{
    const double *part = reinterpret_cast<const double *>(sw + kPartial);
    double a = 0, m = 0, s = 0, q = 0;
    for (int k = threadIdx.x; k < nblocks; k += 32) {
        a += part[4 * k + 0];
        m = fmax(m, part[4 * k + 1]);
        s += part[4 * k + 2];
        q += part[4 * k + 3];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        s += __shfl_xor_sync(0xffffffffu, s, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    }
    if (threadIdx.x == 0) {
        out[0] = P.n ? a / P.n : 0.0;
        out[1] = m;
        out[2] = P.n ? s / P.n : 0.0;
        out[3] = P.n ? q / P.n : 0.0;
    }
}

apbf_status fail(apbf_status st, const std::string &m)
{
    apbf::set_last_error_message(m);
    return st;
}

// The device address of the static scratch array on the current device,
// looked up once per device (the host-side symbol is not a device address).
// The stream must belong to that device: its kernels would otherwise run on
// the stream's device against an address taken on another. A stream that is
// being captured into a graph cannot be asked for its device (the query would
// end the capture), so there the check is skipped, and the first call on the
// device (the lookup, which loads the module) is refused instead of breaking
// the capture.
apbf_status scratch_for_current_device(cudaStream_t stream, uint32_t **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return fail(APBF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 64)
        return fail(APBF_ERR_NOT_SUPPORTED, "device ordinal above 63");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess)
        return fail(APBF_ERR_INVALID_ARG, std::string("cuda_stream: ") + cudaGetErrorString(e));
    if (cap == cudaStreamCaptureStatusNone) {
        int sdev = -1;
        e = cudaStreamGetDevice(stream, &sdev);
        if (e != cudaSuccess)
            return fail(APBF_ERR_INVALID_ARG, std::string("cuda_stream: ") + cudaGetErrorString(e));
        if (sdev != dev)
            return fail(APBF_ERR_INVALID_ARG, "cuda_stream belongs to device " + std::to_string(sdev) +
                                                  ", not to the current device " + std::to_string(dev));
    }
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev] && cap != cudaStreamCaptureStatusNone)
        return fail(APBF_ERR_BAD_STATE, "the first call on a device loads the module: make it outside stream capture");
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_density_scratch);
        if (e != cudaSuccess || !p)
            return fail(APBF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_scratch_ptr[dev];
    return APBF_OK;
}

}  // namespace

extern "C" APBF_API apbf_status apbf_density_stats_static(const float *pos, uint32_t n, float h, float mass,
                                                          float rho0, const float grid_lo[3], const float grid_hi[3],
                                                          double *stats, void *cuda_stream)
{
    if (!stats || !grid_lo || !grid_hi || (n > 0 && !pos))
        return fail(APBF_ERR_INVALID_ARG, "pos, stats, grid_lo and grid_hi must not be NULL");
    if (n > kMaxParticles)
        return fail(APBF_ERR_INVALID_ARG, "n = " + std::to_string(n) + " exceeds the static scratch maximum of " +
                                              std::to_string(kMaxParticles) + " particles");
    if (!(h > 0.0f) || !std::isfinite(h) || !(mass > 0.0f) || !std::isfinite(mass) || !(rho0 > 0.0f) ||
        !std::isfinite(rho0))
        return fail(APBF_ERR_INVALID_ARG, "h, mass and rho0 must be positive and finite");
    Params P{};
    P.n = n;
    P.inv_h = 1.0f / h;
    P.h2 = h * h;
    if (!std::isfinite(P.inv_h) || !(P.h2 > 0.0f))
        return fail(APBF_ERR_INVALID_ARG, "h is too small: 1/h or h*h is not a positive finite float");
    uint64_t ncell = 1;
    int dims[3];
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(grid_lo[a]) || !std::isfinite(grid_hi[a]) || !(grid_lo[a] <= grid_hi[a]))
            return fail(APBF_ERR_INVALID_ARG, "need finite grid_lo <= grid_hi on every axis");
        volatile float ext = grid_hi[a] - grid_lo[a];
        volatile float t = ext * P.inv_h;
        const double fl = std::floor((double)t);
        if (!(fl >= 0.0 && fl < (double)kMaxCells))
            return fail(APBF_ERR_INVALID_ARG, "grid exceeds the static scratch maximum of " +
                                                  std::to_string(kMaxCells) + " cells");
        dims[a] = (int)fl + 1;
        ncell *= (uint64_t)dims[a];
        P.glo[a] = grid_lo[a];
    }
    if (ncell > kMaxCells)
        return fail(APBF_ERR_INVALID_ARG, "grid has " + std::to_string(ncell) +
                                              " cells, above the static scratch maximum of " +
                                              std::to_string(kMaxCells));
    P.nx = dims[0];
    P.ny = dims[1];
    P.nz = dims[2];
    P.ncell = (uint32_t)ncell;
    const double PI = 3.14159265358979323846, hd = h, h2 = hd * hd;
    P.mass_poly6 = (float)((double)mass * 315.0 / (64.0 * PI * std::pow(hd, 9)));
    P.h6 = (float)(h2 * h2 * h2);
    P.rho0 = (double)rho0;

    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint32_t *sw = nullptr;
    apbf_status st = scratch_for_current_device(s, &sw);
    if (st != APBF_OK)
        return st;
    // the cell counts are the only scratch that must start at zero
    cudaError_t e = cudaMemsetAsync(sw + kCount, 0, 4 * (size_t)P.ncell, s);
    const unsigned nb = (n + kSB - 1) / kSB;
    if (e == cudaSuccess && n) {
        hash_count_kernel<<<nb, kSB, 0, s>>>(P, pos, sw);
        start_scan_kernel<<<1, 1024, 0, s>>>(P, sw);
        scatter_index_kernel<<<nb, kSB, 0, s>>>(P, sw);
        rank_copy_kernel<<<nb, kSB, 0, s>>>(P, pos, sw);
        density_scan_kernel<<<nb, kSB, 0, s>>>(P, sw);
    }
    if (e == cudaSuccess) {
        stats_final_kernel<<<1, 32, 0, s>>>(P, sw, (int)nb, stats);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return fail(APBF_ERR_CUDA, std::string("apbf_density_stats_static: ") + cudaGetErrorString(e));
    return APBF_OK;
}
