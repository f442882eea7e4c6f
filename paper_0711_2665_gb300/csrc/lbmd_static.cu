// lbmd_static.cu -- allocation-free variant of the fluid mass/momentum
// reduction: the per-block partial sums live in a file-scope device array
// instead of memory the caller provides.
//
// Who needs it: callers that cannot allocate device memory at the point of
// the call.  Examples are a monitoring loop that runs beside a simulation on
// a GPU whose memory is already fully handed out to another framework's pool,
// and time-critical code that cannot afford cudaMalloc, which implicitly
// synchronises the whole device.  Such a caller passes its populations and
// an output buffer it already owns; this file supplies the scratch.
//
// The array below belongs to this file's own CUDA module.  Under lazy module
// loading (the CUDA default) a module is loaded, and its device arrays are
// allocated, the first time the process uses it on a device: the first call
// of lbmd_population_sums_static on that device.  That first call therefore
// does allocate (and may synchronise); every later call on the device does
// not.  A caller that cannot allocate later makes one call early, before
// handing the GPU's memory to a pool or starting a stream capture.  The
// array then stays allocated until the process exits (or the context is
// reset).  Every call shares it, and it keeps the last call's contents, so
// two calls whose kernels overlap on the GPU (different streams, no ordering
// between them) race on it.
#include "lbmd_internal.cuh"

namespace {

constexpr int SUM_THREADS = 256;
constexpr int SITES_PER_BLOCK = 2048;                // 8 sites per thread
constexpr int MAX_BLOCKS = LBMD_STATIC_SUMS_MAX_SITES / SITES_PER_BLOCK;
constexpr int NPART = 5;                             // rho-1, jx, jy, jz, fluid sites
constexpr size_t PARTIAL_BYTES = sizeof(double) * NPART * MAX_BLOCKS;
constexpr size_t SCRATCH_BYTES = PARTIAL_BYTES + 256;  // + the finished-blocks counter

static_assert(LBMD_STATIC_SUMS_MAX_SITES % SITES_PER_BLOCK == 0, "whole blocks");

// the scratch: block partials, then one counter of finished blocks
static __device__ __align__(256) unsigned char g_sums_scratch[SCRATCH_BYTES];

__global__ void __launch_bounds__(SUM_THREADS) k_population_sums(const float *__restrict__ dev,
                                                                 const uint8_t *__restrict__ solid,
                                                                 int ns, double *out, unsigned char *scratch) {
    using namespace lbmd;
    double *part = reinterpret_cast<double *>(scratch);
    unsigned int *done = reinterpret_cast<unsigned int *>(scratch + PARTIAL_BYTES);
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f, nf = 0.f;
    const int base = blockIdx.x * SITES_PER_BLOCK;
    for (int k = threadIdx.x; k < SITES_PER_BLOCK; k += SUM_THREADS) {
        const int s = base + k;
        if (s >= ns || (solid && solid[s])) continue;
        float m = 0.f, x = 0.f, y = 0.f, z = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float h = __ldg(dev + (size_t)i * ns + s);  // f_i - w_i
            m += h;
            x += (float)cx(i) * h;
            y += (float)cy(i) * h;
            z += (float)cz(i) * h;
        }
        drho += m; jx += x; jy += y; jz += z; nf += 1.f;
    }
    double v[NPART] = {drho, jx, jy, jz, nf};
    __shared__ double red[SUM_THREADS / 32][NPART];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < NPART; ++q) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NPART; ++q) red[warp][q] = v[q];
    __syncthreads();
    __shared__ int am_last;
    if (threadIdx.x == 0) {
        for (int q = 0; q < NPART; ++q) {
            double t = 0.0;
            for (int w = 0; w < SUM_THREADS / 32; ++w) t += red[w][q];
            part[(size_t)blockIdx.x * NPART + q] = t;
        }
        __threadfence();
        am_last = (atomicAdd(done, 1u) == gridDim.x - 1u);
    }
    __syncthreads();
    if (!am_last || threadIdx.x != 0) return;
    __threadfence();
    // the last block adds the partials in block order (same result every call)
    double t[NPART] = {0, 0, 0, 0, 0};
    for (unsigned int b = 0; b < gridDim.x; ++b)
        for (int q = 0; q < NPART; ++q) t[q] += __ldcg(part + (size_t)b * NPART + q);
    out[0] = t[4] + t[0];  // fluid sites x rho_rest (= 1) + sum of deviations
    out[1] = t[1];
    out[2] = t[2];
    out[3] = t[3];
    *done = 0u;
}

}  // namespace

extern "C" lbmd_status lbmd_population_sums_static(const float *dev, const uint8_t *solid, int32_t nx, int32_t ny,
                                                   int32_t nz, double *out, void *stream) {
    if (!dev || !out || nx < 1 || ny < 1 || nz < 1) return LBMD_ERR_INVALID_ARG;
    const double nsd = (double)nx * ny * nz;
    if (nsd > (double)LBMD_STATIC_SUMS_MAX_SITES) return LBMD_ERR_CAPACITY;
    const int ns = nx * ny * nz;
    cudaStream_t st = (cudaStream_t)stream;
    // The array's device address on the current device (a host-side reference
    // to the symbol is not it), looked up on every call: nothing is cached, so
    // a call after cudaDeviceReset (which unloads the module and frees the
    // array) finds the array of the new context.  Once the module is loaded
    // the lookup allocates nothing.
    void *scratch = nullptr;
    if (cudaGetSymbolAddress(&scratch, g_sums_scratch) != cudaSuccess || !scratch) return LBMD_ERR_CUDA;
    // the finished-blocks counter must start at zero; the partials are all
    // overwritten by this call
    if (cudaMemsetAsync((unsigned char *)scratch + PARTIAL_BYTES, 0, sizeof(unsigned int), st) != cudaSuccess)
        return LBMD_ERR_CUDA;
    const int blocks = (ns + SITES_PER_BLOCK - 1) / SITES_PER_BLOCK;
    k_population_sums<<<blocks, SUM_THREADS, 0, st>>>(dev, solid, ns, out, (unsigned char *)scratch);
    return cudaGetLastError() == cudaSuccess ? LBMD_OK : LBMD_ERR_CUDA;
}
