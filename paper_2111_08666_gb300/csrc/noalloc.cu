// Diagnostics of populations held in the public layout, computed without
// allocating any memory.
//
// Some callers cannot call cudaMalloc, or let a library call it on their
// behalf: for instance a process whose device memory is all handed out by
// its own pool allocator, or a time-critical loop that must not allocate
// once it has started.  mclbm_diagnostics needs a lattice (whose creation
// allocates) and keeps its per-block partial sums in memory the lattice
// owns.  This entry point takes the populations and the solid mask in
// caller-owned device memory and keeps its partial sums in a fixed array in
// the library's own device globals instead.
//
// The array has room for NOALLOC_BLOCKS blocks of partial sums; each block
// reduces NOALLOC_NODES_PER_BLOCK nodes, so lattices of up to
// NOALLOC_MAX_NODES nodes are accepted and larger ones are rejected.  Every
// device that loads the library holds the array (64 KB) until the process
// exits.  All calls share it: calls that overlap on the GPU (on different
// streams, or from different threads) race on it and must be serialised by
// the caller.  Every call rewrites every partial it reads, so nothing left
// by an earlier call affects a later one.
#include <cmath>
#include <mutex>
#include <string>

#include "lbm.cuh"

namespace mclbm {

namespace {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_NODES_PER_THREAD = 16;
constexpr int NOALLOC_NODES_PER_BLOCK = NOALLOC_THREADS * NOALLOC_NODES_PER_THREAD;
constexpr int NOALLOC_BLOCKS = 1024;
constexpr long long NOALLOC_MAX_NODES = (long long)NOALLOC_BLOCKS * NOALLOC_NODES_PER_BLOCK;
constexpr int NOALLOC_ACC = 8;
constexpr int NOALLOC_MAX_DEVICES = 64;

// per-block partial sums, then the 8 results
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_BLOCKS * NOALLOC_ACC + 8];

// Device address of g_noalloc_scratch per device ordinal.  In host code the
// symbol name stands for a host-side shadow, not for device memory, so the
// address must come from cudaGetSymbolAddress with the device current.
double *g_scratch_addr[NOALLOC_MAX_DEVICES] = {};
std::mutex g_scratch_mutex;

__device__ __forceinline__ double noalloc_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Pass 1: block b reduces nodes [b * NODES_PER_BLOCK, (b+1) * NODES_PER_BLOCK).
//   acc[0] mass1  acc[1] mass2  acc[2] fluid nodes  acc[3] water nodes
//   acc[4] P_in sum  acc[5] P_in count  acc[6] P_out sum  acc[7] P_out count
// (A non-finite density shows in the results themselves: the masses and
// saturations it enters become NaN or infinite.)
__global__ void __launch_bounds__(NOALLOC_THREADS)
    noalloc_partial_kernel(const double *f, const uint8_t *solid, int nx, int ny, double g_coh,
                           int periodic_y, double *scratch) {
    double acc[NOALLOC_ACC];
#pragma unroll
    for (int k = 0; k < NOALLOC_ACC; ++k) acc[k] = 0.0;
    const long long n = (long long)nx * ny;
    const long long first = (long long)blockIdx.x * NOALLOC_NODES_PER_BLOCK;
    for (int j = 0; j < NOALLOC_NODES_PER_THREAD; ++j) {
        const long long k = first + (long long)j * NOALLOC_THREADS + threadIdx.x;
        if (k >= n) break;
        if (solid[k]) continue;
        const int x = (int)(k % nx), y = (int)(k / nx);
        double r1 = 0.0, r2 = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            r1 += f[(long long)i * n + k];
            r2 += f[(long long)(9 + i) * n + k];
        }
        acc[0] += r1;
        acc[1] += r2;
        acc[2] += 1.0;
        acc[3] += (r2 > r1) ? 1.0 : 0.0;
        if (x == 0 || x == nx - 1) {
            // boundary pressure away from walls: no solid within 2 rows
            bool site = true;
            for (int d = -2; d <= 2 && site; ++d) {
                int yy = y + d;
                if (yy < 0 || yy >= ny) {
                    if (!periodic_y) {
                        site = false;
                        break;
                    }
                    yy = (yy + ny) % ny;
                }
                if (solid[(long long)yy * nx + x]) site = false;
            }
            if (site) {
                const int o = x == 0 ? 4 : 6;
                acc[o] += (r1 + r2) / 3.0 + g_coh / 3.0 * r1 * r2;  // Eq. 14
                acc[o + 1] += 1.0;
            }
        }
    }
    __shared__ double red[NOALLOC_THREADS / 32][NOALLOC_ACC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NOALLOC_ACC; ++k) {
        const double v = noalloc_warp_sum(acc[k]);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NOALLOC_ACC) {
        double s = 0.0;
        for (int w = 0; w < NOALLOC_THREADS / 32; ++w) s += red[w][threadIdx.x];
        scratch[blockIdx.x * NOALLOC_ACC + threadIdx.x] = s;
    }
}

// Pass 2: add the partials in block order (deterministic), form the 8
// results in the scratch tail and, if given, in a device output.
__global__ void noalloc_final_kernel(double *scratch, int nblocks, double *out_dev) {
    __shared__ double tot[NOALLOC_ACC];
    if (threadIdx.x < NOALLOC_ACC) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += scratch[b * NOALLOC_ACC + threadIdx.x];
        tot[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000ULL);
        double r[8];
        r[0] = tot[0];
        r[1] = tot[1];
        r[2] = tot[2] > 0 ? tot[3] / tot[2] : nan;
        r[3] = (tot[0] + tot[1]) > 0 ? tot[1] / (tot[0] + tot[1]) : nan;
        r[4] = tot[5] > 0 ? tot[4] / tot[5] : nan;
        r[5] = tot[7] > 0 ? tot[6] / tot[7] : nan;
        r[6] = r[4] - r[5];
        r[7] = tot[2];
        double *res = scratch + NOALLOC_BLOCKS * NOALLOC_ACC;
        for (int k = 0; k < 8; ++k) {
            res[k] = r[k];
            if (out_dev) out_dev[k] = r[k];
        }
    }
}

bool noalloc_is_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Set-up, once per device, with that device current.
int scratch_for_current_device(double **ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return fail(MCLBM_ERR_ARG, "device ordinal beyond the static scratch table");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *ptr = g_scratch_addr[dev];
    return MCLBM_OK;
}

}  // namespace

}  // namespace mclbm

using namespace mclbm;

extern "C" int mclbm_diagnostics_noalloc(const double *f, const uint8_t *solid, int nx, int ny,
                                         double g_coh, int periodic_y, double *out,
                                         void *cuda_stream) {
    if (!f || !solid || !out) return fail(MCLBM_ERR_ARG, "f, solid and out must not be NULL");
    if (nx < 1 || ny < 1) return fail(MCLBM_ERR_ARG, "nx and ny must be >= 1");
    const long long n = (long long)nx * ny;
    if (n > NOALLOC_MAX_NODES)
        return fail(MCLBM_ERR_ARG, "lattice of " + std::to_string(n) +
                                       " nodes exceeds the static scratch of "
                                       "mclbm_diagnostics_noalloc (at most " +
                                       std::to_string(NOALLOC_MAX_NODES) +
                                       " nodes); use mclbm_diagnostics");
    if (!std::isfinite(g_coh)) return fail(MCLBM_ERR_ARG, "g_coh must be finite");
    if (!noalloc_is_device(f) || !noalloc_is_device(solid))
        return fail(MCLBM_ERR_ARG, "f and solid must be device memory");
    double *scratch = nullptr;
    if (int rc = scratch_for_current_device(&scratch)) return rc;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    const bool out_dev = noalloc_is_device(out);
    const int nblocks = (int)((n + NOALLOC_NODES_PER_BLOCK - 1) / NOALLOC_NODES_PER_BLOCK);
    noalloc_partial_kernel<<<nblocks, NOALLOC_THREADS, 0, stream>>>(f, solid, nx, ny, g_coh,
                                                                   periodic_y ? 1 : 0, scratch);
    noalloc_final_kernel<<<1, 32, 0, stream>>>(scratch, nblocks, out_dev ? out : nullptr);
    count_launch(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "diagnostics kernels");
    if (!out_dev) {
        e = cudaMemcpyAsync(out, scratch + NOALLOC_BLOCKS * NOALLOC_ACC, 8 * sizeof(double),
                            cudaMemcpyDeviceToHost, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(results)");
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    return MCLBM_OK;
}
