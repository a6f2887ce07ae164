// solve_static.cu -- sfft_solve_static: the solve of M theta = rhs (Eq. 18)
// on a workspace held in a file-scope device array, so that no call
// allocates memory.
//
// The array holds SFFT_SOLVE_STATIC_MAX_N^2 doubles twice (the scaled matrix
// A and W = L^-1) plus 256 KiB for the vectors: 16.25 MiB per device, owned
// by this translation unit's module and placed by the CUDA driver when the
// module is loaded.  Each call lays the workspace for its own n out from the
// start of the array.  Nothing in it has to start at zero: the solve kernel
// first resets the status flags and statistics, and it writes every element
// of A, W and the vectors before it reads them.  Two calls whose executions overlap on one device (different
// streams, or host threads without ordering) share the array and race.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kMaxN = SFFT_SOLVE_STATIC_MAX_N;
constexpr int kMaxGrid = sfft::kMaxSolveGrid;  // per-block partial sums: 2 doubles per block
constexpr int kMaxDevices = 64;  // devices with their own setup record
constexpr size_t kAlign = 256;
constexpr size_t kScratchBytes = 2 * kMaxN * kMaxN * sizeof(double) + 256 * 1024;

}  // namespace

static __device__ __align__(256) unsigned char sfft_static_scratch[kScratchBytes];

namespace {

// One record per device: the array's device address and the cooperative grid
// of the solve kernel for each compute type, set up once.
struct DeviceState {
    std::atomic<int> ready{0};
    unsigned char *base = nullptr;
    int grid[2] = {0, 0};  // [0] FP32, [1] FP64
};

DeviceState g_dev[kMaxDevices];
std::mutex g_setup;

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return SFFT_OK;
    if (e == cudaErrorMemoryAllocation) return SFFT_ERR_OOM;
    return SFFT_ERR_CUDA;
}

// Setup for the current device `dev`: the array's address (loading the
// module if it is not yet loaded) and the grid sizes.  Thread-safe.
int device_state(int dev, DeviceState **out) {
    DeviceState &d = g_dev[dev];
    if (!d.ready.load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> lock(g_setup);
        if (!d.ready.load(std::memory_order_relaxed)) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, sfft_static_scratch);
            if (e != cudaSuccess) return status_of(e);
            const int g32 = sfft::solve_grid_size(false), g64 = sfft::solve_grid_size(true);
            if (g32 <= 0 || g32 > kMaxGrid || g64 <= 0 || g64 > kMaxGrid) return SFFT_ERR_UNSUPPORTED;
            d.base = static_cast<unsigned char *>(p);
            d.grid[0] = g32;
            d.grid[1] = g64;
            d.ready.store(1, std::memory_order_release);
        }
    }
    *out = &d;
    return SFFT_OK;
}

}  // namespace

int sfft_solve_static(const double *d_M, const double *d_rhs, int32_t n, int32_t precision, double *d_x,
                      sfft_solve_info *d_info, sfft_stream_t stream) {
    if (!d_M || !d_rhs || !d_x) return SFFT_ERR_INVALID;
    if (precision != SFFT_PREC_FP64 && precision != SFFT_PREC_MIXED) return SFFT_ERR_INVALID;
    if (n < 1) return SFFT_ERR_INVALID;
    if ((size_t)n > kMaxN) return SFFT_ERR_UNSUPPORTED;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return status_of(e);
    if (dev < 0 || dev >= kMaxDevices) return SFFT_ERR_UNSUPPORTED;
    DeviceState *d = nullptr;
    const int st = device_state(dev, &d);
    if (st != SFFT_OK) return st;

    const bool fp64 = precision == SFFT_PREC_FP64;
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    const size_t nn = (size_t)n;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char *q = d->base + off;
        off += (bytes + kAlign - 1) / kAlign * kAlign;
        return q;
    };
    sfft::SolveBuffers b;
    b.n = n;
    b.fp64 = fp64;
    b.grid = d->grid[fp64 ? 1 : 0];
    b.A = take(nn * nn * rsz);
    b.W = take(nn * nn * rsz);
    b.zv = take(sfft::solve_vec_elems(n) * rsz);
    b.dsc = reinterpret_cast<double *>(take(nn * sizeof(double)));
    b.r = reinterpret_cast<double *>(take(nn * sizeof(double)));
    b.xw = reinterpret_cast<double *>(take((nn + 8 + 2 * kMaxGrid) * sizeof(double)));
    b.flag = reinterpret_cast<int *>(take(4 * sizeof(int)));
    if (off > kScratchBytes) return SFFT_ERR_UNSUPPORTED;  // not reached for n <= SFFT_SOLVE_STATIC_MAX_N
    e = sfft::solve_on_buffers(b, d_M, d_rhs, d_x, d_info, (cudaStream_t)stream);
    return status_of(e);
}
