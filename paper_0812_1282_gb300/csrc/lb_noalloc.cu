// Diagnostics reduction that allocates nothing (lb_stats_noalloc).
//
// Some callers cannot allocate device memory at the moment they need the
// numbers: an application that owns every byte of the device through its
// own memory pool and forbids stray cudaMalloc calls, or a long-running
// service that must not fragment or grow its memory footprint mid-run.  For
// them this file offers a variant of the moments reduction whose scratch
// space is a fixed, file-scope device array instead of a buffer from the
// library's workspace.
//
// The array (kMaxBlocks block partials of kFields doubles, 48 KiB) is created
// when the library is loaded on a device and lives until the process exits.
// Its device address is looked up once per device, on the first call for
// that device (the device holding the population arrays).  Every call
// shares the array: two calls
// whose kernels overlap on the GPU (different streams, no ordering between
// them) race on it and may return wrong numbers; calls ordered on one
// stream are safe.  Each call writes every slot it later reads, so nothing
// has to be cleared first.
//
// The kernels are launched with cudaLaunchKernel, whose return value is the
// launch's own status: the runtime's per-thread "last error" is neither read
// nor cleared, so an error left there by an earlier, unrelated call stays
// for its owner and is not reported as a failure of this one.  The caller's
// current device is restored before returning.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>

#include "../../include/lbfe.h"

namespace {

constexpr int kFields = 6;       // mass, order, mom_x, mom_y, max_u, nonfinite
constexpr int kBlock = 256;      // threads per block
constexpr int kMaxBlocks = 1024; // block partials the scratch array holds
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kMaxBlocks * kFields];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

__device__ __forceinline__ void reduce_warp(double (&v)[kFields])
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < kFields; ++k) {
            const double o = __shfl_xor_sync(0xffffffffu, v[k], off);
            v[k] = (k == 4) ? fmax(v[k], o) : v[k] + o;
        }
}

// Block-level combine of per-thread partial sums; result valid in thread 0.
__device__ __forceinline__ void reduce_block(double (&v)[kFields])
{
    __shared__ double part[kBlock / 32][kFields];
    reduce_warp(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < kFields; ++k) part[wid][k] = v[k];
    __syncthreads();
    if (wid == 0) {
        for (int k = 0; k < kFields; ++k) v[k] = lane < (blockDim.x >> 5) ? part[lane][k] : 0.0;
        reduce_warp(v);
    }
}

// Pass 1: each block reduces a grid-stride share of the nodes of absolute
// populations f, g ([9][n] arrays) into scratch[blockIdx.x].
template <typename T>
__global__ void __launch_bounds__(kBlock) noalloc_partials(const T* __restrict__ f,
                                                           const T* __restrict__ g, long long n,
                                                           double* __restrict__ scratch)
{
    double acc[kFields] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        double fv[9], ph = 0.0, rho = 0.0;
        for (int i = 0; i < 9; ++i) {
            fv[i] = double(f[i * n + k]);
            rho += fv[i];
            ph += double(g[i * n + k]);
        }
        // e_i in the order 0, (1,0), (-1,0), (0,1), (0,-1), (1,1), (-1,-1), (-1,1), (1,-1)
        const double jx = (fv[1] - fv[2]) + (fv[5] - fv[6]) + (fv[8] - fv[7]);
        const double jy = (fv[3] - fv[4]) + (fv[5] - fv[6]) + (fv[7] - fv[8]);
        const double um = sqrt(jx * jx + jy * jy) / rho;
        const bool ok = isfinite(rho) && isfinite(ph) && isfinite(um);
        acc[0] += rho;
        acc[1] += ph;
        acc[2] += jx;
        acc[3] += jy;
        acc[4] = ok ? fmax(acc[4], um) : acc[4];
        acc[5] += ok ? 0.0 : 1.0;
    }
    reduce_block(acc);
    if (threadIdx.x == 0)
        for (int k = 0; k < kFields; ++k) scratch[blockIdx.x * kFields + k] = acc[k];
}

// Pass 2: one block combines the partials (fixed order) into the output.
__global__ void __launch_bounds__(kBlock) noalloc_finish(const double* __restrict__ scratch,
                                                         int nblocks, double* __restrict__ out)
{
    double acc[kFields] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < kFields; ++k) {
            const double v = scratch[b * kFields + k];
            acc[k] = (k == 4) ? fmax(acc[k], v) : acc[k] + v;
        }
    reduce_block(acc);
    if (threadIdx.x == 0)
        for (int k = 0; k < kFields; ++k) out[k] = acc[k];
}

// Device address of the scratch array for the current device, looked up
// once per device.
cudaError_t scratch_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_scratch_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Restores the calling thread's current device when it goes out of scope.
struct DeviceRestore {
    int prev = -1;
    ~DeviceRestore()
    {
        int now = -1;
        if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
    }
};

// Device that holds `p` (device memory only), or -1.
int device_of(const void* p)
{
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess || attr.type != cudaMemoryTypeDevice)
        return -1;
    return attr.device;
}

}  // namespace

extern "C" int lb_stats_noalloc(const void* f, const void* g, int nx, int ny, int precision,
                                double* stats_dev, void* stream)
{
    if (!f || !g || !stats_dev) return LB_ERR_INVALID_ARG;
    if (precision != LB_FP32 && precision != LB_FP64) return LB_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1) return LB_ERR_INVALID_ARG;
    long long n = (long long)nx * ny;
    if (9 * n > INT_MAX) return LB_ERR_INVALID_ARG;  // beyond LB_STATS_NOALLOC_MAX_VALUES
    // all three arrays on one device; the work runs there
    const int dev = device_of(f);
    if (dev < 0 || device_of(g) != dev || device_of(stats_dev) != dev) return LB_ERR_INVALID_ARG;
    DeviceRestore restore;
    if (cudaGetDevice(&restore.prev) != cudaSuccess) return LB_ERR_CUDA;
    if (dev != restore.prev && cudaSetDevice(dev) != cudaSuccess) return LB_ERR_CUDA;
    double* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return LB_ERR_CUDA;
    int blocks = int(std::min<long long>((n + kBlock - 1) / kBlock, kMaxBlocks));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* pass1[] = {(void*)&f, (void*)&g, &n, &scratch};
    const void* k1 = precision == LB_FP32 ? reinterpret_cast<const void*>(&noalloc_partials<float>)
                                          : reinterpret_cast<const void*>(&noalloc_partials<double>);
    if (cudaLaunchKernel(k1, dim3(blocks), dim3(kBlock), pass1, 0, s) != cudaSuccess)
        return LB_ERR_CUDA;
    void* pass2[] = {&scratch, &blocks, &stats_dev};
    if (cudaLaunchKernel(reinterpret_cast<const void*>(&noalloc_finish), dim3(1), dim3(kBlock),
                         pass2, 0, s) != cudaSuccess)
        return LB_ERR_CUDA;
    return LB_OK;
}
