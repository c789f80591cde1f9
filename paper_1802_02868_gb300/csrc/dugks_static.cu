// dugks_static.cu -- an allocation-free variant of the FP64 conservation
// reduction (sum |V| phi and sum |V| rho over one mesh).
//
// dugks_conservation() reduces through per-tile partial sums that live in
// device memory the simulation allocated with cudaMalloc.  Some callers cannot
// allocate device memory at all, for example a host loop that runs under a
// device-memory budget owned by another allocator (such as PyTorch's caching
// allocator, which may already hold all free memory, so a cudaMalloc can fail
// or fragment it), or a latency-critical loop in which the implicit device
// synchronisation of cudaMalloc/cudaFree is not acceptable.  For them,
// dugks_conservation_static() takes caller-owned device buffers and keeps its
// scratch (one partial pair per block) in the file-scope array below, which
// every GPU that loads this library holds until the process exits.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "../../include/dugks.h"

namespace {

constexpr int kThreads = 256;
constexpr int kCellsPerThread = 16;
constexpr int kCellsPerBlock = kThreads * kCellsPerThread;   // 4096

}  // namespace

// Scratch: one (sum |V| phi, sum |V| rho) pair per block, 64 KiB per device.
static __device__ __align__(256) double2 dugks_static_partials[DUGKS_STATIC_MAX_CELLS / 4096];

namespace {

static_assert(DUGKS_STATIC_MAX_CELLS % kCellsPerBlock == 0, "scratch sizing");
constexpr int kMaxBlocks = DUGKS_STATIC_MAX_CELLS / kCellsPerBlock;

__device__ __forceinline__ double2 block_sum(double a, double b)
{
    __shared__ double2 red[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = make_double2(a, b);
    __syncthreads();
    double2 s = make_double2(0.0, 0.0);
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; w++) { s.x += red[w].x; s.y += red[w].y; }
    return s;
}

// Block b sums the cells [b * 4096, (b + 1) * 4096) of the dense field and
// writes its pair to partials[b]; every used slot is overwritten, so nothing
// needs clearing between calls.
__global__ void __launch_bounds__(kThreads) k_cons_partial(const double *__restrict__ phi, const double *__restrict__ dx,
                                                           const double *__restrict__ dy, int nx, long long n,
                                                           double rhoB, double drho, double phiB, double2 *partials)
{
    const long long base = (long long)blockIdx.x * kCellsPerBlock;
    double a = 0.0, b = 0.0;
    for (int k = 0; k < kCellsPerThread; k++) {
        const long long c = base + (long long)k * kThreads + threadIdx.x;
        if (c < n) {
            const int i = (int)(c % nx), j = (int)(c / nx);
            const double vol = dx[i] * dy[j];
            const double v = phi[c];
            a += vol * v;
            b += vol * (rhoB + drho * (v - phiB));
        }
    }
    const double2 s = block_sum(a, b);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// One block adds the partials in a fixed order and writes out[0], out[1].
__global__ void __launch_bounds__(kThreads) k_cons_final(const double2 *__restrict__ partials, int nblocks, double *out)
{
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += kThreads) {
        a += partials[k].x;
        b += partials[k].y;
    }
    const double2 s = block_sum(a, b);
    if (threadIdx.x == 0) {
        out[0] = s.x;
        out[1] = s.y;
    }
}

constexpr int kMaxDevices = 64;
std::atomic<double2 *> g_scratch[kMaxDevices];
std::mutex g_setup;

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the array's name as a device address).
int scratch_address(double2 **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DUGKS_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return DUGKS_ERR_UNSUPPORTED;
    double2 *p = g_scratch[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lock(g_setup);
        p = g_scratch[dev].load(std::memory_order_relaxed);
        if (!p) {
            void *addr = nullptr;
            if (cudaGetSymbolAddress(&addr, dugks_static_partials) != cudaSuccess) return DUGKS_ERR_CUDA;
            p = (double2 *)addr;
            g_scratch[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return DUGKS_OK;
}

}  // namespace

extern "C" int dugks_conservation_static(const double *phi, const double *dx, const double *dy, int nx, int ny,
                                         double phiA, double phiB, double rhoA, double rhoB, double *out,
                                         void *cuda_stream)
{
    if (!phi || !dx || !dy || !out || nx < 1 || ny < 1) return DUGKS_ERR_ARG;
    const long long n = (long long)nx * ny;
    if (n > DUGKS_STATIC_MAX_CELLS) return DUGKS_ERR_ARG;
    if (phiA == phiB) return DUGKS_ERR_ARG;
    double2 *partials = nullptr;
    int rc = scratch_address(&partials);
    if (rc) return rc;
    const int nblocks = (int)((n + kCellsPerBlock - 1) / kCellsPerBlock);
    if (nblocks > kMaxBlocks) return DUGKS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const double drho = (rhoA - rhoB) / (phiA - phiB);
    k_cons_partial<<<nblocks, kThreads, 0, st>>>(phi, dx, dy, nx, n, rhoB, drho, phiB, partials);
    k_cons_final<<<1, kThreads, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError() == cudaSuccess ? DUGKS_OK : DUGKS_ERR_CUDA;
}
