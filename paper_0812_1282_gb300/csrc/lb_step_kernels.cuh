// Fused step kernels (single domain and batched work list) and their
// launchers, templated on precision, collision and the strip width.
//
// The strip width W = 32 NW is a template constant (NWC = NW) for the three
// widths the autotuner uses (64, 128, 256 columns), so every shared-memory
// offset of the stage ring and the phi rings folds into an immediate; other
// widths (multiples of 32 up to 256) take the generic form (NWC = 0, width
// read from blockDim).  Both forms run the same code on the same data.
#pragma once

#include <cuda_runtime.h>

#include "lb_internal.h"
#include "lb_step.cuh"
#include "lb_step_compact.cuh"

namespace lbfe {

// Stage-ring depth: rows of bulk copies in flight per CTA.
template <typename Real>
constexpr int kStages = sizeof(Real) == 4 ? 4 : 3;
// Named barrier of the compute warps of the batched full-storage form.
constexpr int kComputeBarrierFull = 1;

// Launch shape: blockDim.x = W + 32 (one producer warp, W / 32 compute
// warps), W the strip width.
// Row bands of a single-domain launch: the CTAs of grid row g take band
// (g band_mul) mod gridDim.y (band_mul coprime to it, 1 = in order), so that
// the host can make vertically adjacent bands start about one band's
// duration apart: a band's first rows are then read while its lower
// neighbour reads the same rows as its last, and come from L2.
__device__ __forceinline__ int band_of(int band_mul)
{
    return band_mul > 1 ? int((long long)blockIdx.y * band_mul % gridDim.y) : int(blockIdx.y);
}

template <typename Real, bool MRT, int NWC>
__global__ void __launch_bounds__(288) step_single_kernel(DomDesc D, int parity, int rows,
                                                          int band_mul)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int S = kStages<Real>;
    const int NW = NWC > 0 ? NWC : int(blockDim.x >> 5) - 1;
    init_stages<Real, S, NWC>(smem, NW);
    const int warp = int(threadIdx.x >> 5);
    const int x0 = blockIdx.x * 32 * NW, y0 = band_of(band_mul) * rows;
    unsigned q = 0;
    if (warp == 0) {
        produce_tile<Real, S, NWC>(D, parity, x0, y0, rows, smem, NW, q);
        drain_stages<Real, S, NWC>(smem, NW, q, D.err);
    } else {
        consume_tile<Real, MRT, S, NWC>(D, parity, x0, y0, rows, smem, NW, warp - 1, q);
    }
}

// Persistent form: a fixed grid walks a list of tiles of many domains.  The
// producer warp takes the next tile from a device counter (dynamic load
// balance: tiles differ in size) and names it to the compute warps through
// the tile's first stage slot; the stage ring carries over from tile to
// tile.  sched[0] is the tile counter, sched[1] counts finished CTAs; the
// last CTA to finish resets both for the next launch.
template <typename Real, bool MRT, int NWC>
__global__ void __launch_bounds__(288) step_batch_kernel(const DomDesc* __restrict__ descs,
                                                         const WorkItem* __restrict__ items,
                                                         int n_items, int parity, int* sched,
                                                         unsigned* err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int tags[kStages<Real>];
    __shared__ NodeParams<Real> tile_prm;  // the current tile's node parameters
    constexpr int S = kStages<Real>;
    const int NW = NWC > 0 ? NWC : int(blockDim.x >> 5) - 1;
    init_stages<Real, S, NWC>(smem, NW);
    const int warp = int(threadIdx.x >> 5), lane = int(threadIdx.x & 31);
    unsigned q = 0;
    if (warp == 0) {
        for (;;) {
            int it = 0;
            if (lane == 0) it = atomicAdd(sched, 1);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it >= n_items) {
                produce_end<Real, S, NWC>(smem, NW, q, tags, err);
                break;
            }
            const WorkItem w = items[it];
            const DomDesc D = descs[w.dom];
            produce_tile<Real, S, NWC>(D, parity, w.x0, w.y0, w.rows, smem, NW, q, tags, it);
        }
        drain_stages<Real, S, NWC>(smem, NW, q, err);
        if (lane == 0) {
            __threadfence();
            if (atomicAdd(sched + 1, 1) == int(gridDim.x) - 1) {  // last CTA: reset
                sched[0] = 0;
                sched[1] = 0;
                __threadfence();
            }
        }
    } else {
        for (;;) {
            const int it = next_tag<Real, S, NWC>(smem, NW, q, tags, err);
            // one decision for all compute warps (the end of the list, or a
            // failed wait on any of them), so that they meet at the same
            // barriers
            if (named_sync_or(kComputeBarrierFull, 32 * NW, it < 0 || it >= n_items)) break;
            const WorkItem w = items[it];
            const DomDesc D = descs[w.dom];
            // every compute warp is past the previous tile: refresh the shared
            // copy of the node parameters, which the collision reads at each use
            if (warp == 1 && lane == 0) tile_prm = node_params<Real>(D);
            named_sync(kComputeBarrierFull, 32 * NW);
            consume_tile<Real, MRT, S, NWC>(D, parity, w.x0, w.y0, w.rows, smem, NW, warp - 1, q,
                                            &tile_prm);
        }
    }
}

// Compact-g forms (FP32, tau_phi = 1; lb_step_compact.cuh).  Same launch
// shapes and scheduling as above, with strips of compact_strip(bx) columns.
template <bool MRT, int NWC>
__global__ void __launch_bounds__(320) step_single_compact_kernel(DomDesc D, int parity, int rows,
                                                                  int band_mul)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int S = kStagesC;
    const int NW = NWC > 0 ? NWC : int(blockDim.x >> 5) - 1;
    init_stages_c<S>(smem, NW);
    const int warp = int(threadIdx.x >> 5);
    const int x0 = blockIdx.x * compact_strip(32 * NW), y0 = band_of(band_mul) * rows;
    unsigned q = 0;
    if (warp == 0) {
        produce_tile_c<S, NWC>(D, parity, x0, y0, rows, 0, smem, NW, q);
        drain_stages<float, S, NWC>(smem, NW, q, D.err);
    } else {
        consume_tile_c<MRT, S, NWC>(D, parity, x0, y0, rows, 0, smem, NW, warp - 1, q);
    }
}

// Register budget of the batched compact kernel: 96 registers per thread,
// so that as many CTAs fit an SM as their shared memory allows (four of
// NW = 4).
template <bool MRT, int NWC>
__global__ void __maxnreg__(96)
    step_batch_compact_kernel(const DomDesc* __restrict__ descs,
                                                                 const WorkItem* __restrict__ items,
                                                                 int n_items, int parity,
                                                                 int* sched, unsigned* err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int tags[kStagesC];
    __shared__ NodeParams<float> tile_prm;  // the current tile's node parameters
    __shared__ DomDesc tile_desc;           // and its domain (compute warps)
    constexpr int S = kStagesC;
    const int NW = NWC > 0 ? NWC : int(blockDim.x >> 5) - 1;
    init_stages_c<S>(smem, NW);
    const int warp = int(threadIdx.x >> 5), lane = int(threadIdx.x & 31);
    unsigned q = 0;
    if (warp == 0) {
        for (;;) {
            int it = 0;
            if (lane == 0) it = atomicAdd(sched, 1);
            it = __shfl_sync(0xffffffffu, it, 0);
            if (it >= n_items) {
                produce_end<float, S, NWC>(smem, NW, q, tags, err);
                break;
            }
            const WorkItem w = items[it];
            const DomDesc D = descs[w.dom];
            produce_tile_c<S, NWC>(D, parity, w.x0, w.y0, w.rows, w.cols, smem, NW, q, tags, it);
        }
        drain_stages<float, S, NWC>(smem, NW, q, err);
        if (lane == 0) {
            __threadfence();
            if (atomicAdd(sched + 1, 1) == int(gridDim.x) - 1) {
                sched[0] = 0;
                sched[1] = 0;
                __threadfence();
            }
        }
    } else {
        for (;;) {
            const int it = next_tag<float, S, NWC>(smem, NW, q, tags, err);
            // one decision for all compute warps (a failed wait on one of
            // them stops all), so that they meet at the same barriers
            if (named_sync_or(kComputeBarrier, 32 * NW, it < 0 || it >= n_items)) break;
            const WorkItem w = items[it];
            // every compute warp is past the previous tile: refresh the shared
            // copies of the domain descriptor and its node parameters, which
            // the tile reads at each use instead of holding them in registers
            if (warp == 1 && lane == 0) {
                tile_desc = descs[w.dom];
                tile_prm = node_params<float>(tile_desc);
            }
            named_sync(kComputeBarrier, 32 * NW);
            consume_tile_c<MRT, S, NWC, true>(tile_desc, parity, w.x0, w.y0, w.rows, w.cols, smem,
                                              NW, warp - 1, q, &tile_prm,
                                              (w.flags & kItemSeal) != 0);
        }
    }
}

template <bool MRT, int NWC>
cudaError_t launch_step_compact_t(const DomDesc& d, const DomDesc* d_descs,
                                  const WorkItem* d_items, int n_items, int n_dom, int parity,
                                  int bx, int rows, int band_mul, int grid_p, int* sched, cudaStream_t s)
{
    const size_t smem = StageLayoutC(bx / 32, kStagesC).total();
    const int threads = bx + 32;
    if (n_dom == 1 && d_items == nullptr) {
        const int w = compact_strip(bx);
        dim3 grid((d.nx + w - 1) / w, (d.ny + rows - 1) / rows);
        step_single_compact_kernel<MRT, NWC><<<grid, threads, smem, s>>>(d, parity, rows,
                                                                        band_mul);
    } else {
        const int grid = grid_p > 0 ? grid_p : n_items;
        step_batch_compact_kernel<MRT, NWC><<<grid, threads, smem, s>>>(d_descs, d_items, n_items,
                                                                        parity, sched, d.err);
    }
    return cudaGetLastError();
}

template <typename Real, bool MRT, int NWC>
cudaError_t launch_step_t(const DomDesc& d, const DomDesc* d_descs, const WorkItem* d_items,
                          int n_items, int n_dom, int parity, int bx, int rows, int band_mul, int grid_p,
                          int* sched, cudaStream_t s)
{
    const size_t smem = StageLayout<Real>(bx / 32, kStages<Real>).total();
    const int threads = bx + 32;
    if (n_dom == 1 && d_items == nullptr) {
        dim3 grid((d.nx + bx - 1) / bx, (d.ny + rows - 1) / rows);
        step_single_kernel<Real, MRT, NWC><<<grid, threads, smem, s>>>(d, parity, rows, band_mul);
    } else {
        const int grid = grid_p > 0 ? grid_p : n_items;
        step_batch_kernel<Real, MRT, NWC><<<grid, threads, smem, s>>>(d_descs, d_items, n_items,
                                                                      parity, sched, d.err);
    }
    return cudaGetLastError();
}

// one_body: a batched launch takes the kernel built for any width (NW read
// from the block size) instead of the one built for its own width.  The
// classes of a schedule run side by side on the SMs, and with one body they
// share the instruction caches.
template <bool MRT>
cudaError_t launch_step_compact_w(const DomDesc& d, const DomDesc* d_descs,
                                  const WorkItem* d_items, int n_items, int n_dom, int parity,
                                  int bx, int rows, int band_mul, int grid_p, int* sched,
                                  bool one_body, cudaStream_t s)
{
    if (one_body && !(n_dom == 1 && d_items == nullptr))
        return launch_step_compact_t<MRT, 0>(d, d_descs, d_items, n_items, n_dom, parity, bx,
                                             rows, band_mul, grid_p, sched, s);
    switch (bx) {
        case 32:
            return launch_step_compact_t<MRT, 1>(d, d_descs, d_items, n_items, n_dom, parity, bx,
                                                 rows, band_mul, grid_p, sched, s);
        case 96:
            return launch_step_compact_t<MRT, 3>(d, d_descs, d_items, n_items, n_dom, parity, bx,
                                                 rows, band_mul, grid_p, sched, s);
        case 64:
            return launch_step_compact_t<MRT, 2>(d, d_descs, d_items, n_items, n_dom, parity, bx,
                                                 rows, band_mul, grid_p, sched, s);
        case 128:
            return launch_step_compact_t<MRT, 4>(d, d_descs, d_items, n_items, n_dom, parity, bx,
                                                 rows, band_mul, grid_p, sched, s);
        case 256:
            return launch_step_compact_t<MRT, 8>(d, d_descs, d_items, n_items, n_dom, parity, bx,
                                                 rows, band_mul, grid_p, sched, s);
        default:
            return launch_step_compact_t<MRT, 0>(d, d_descs, d_items, n_items, n_dom, parity, bx,
                                                 rows, band_mul, grid_p, sched, s);
    }
}

template <typename Real, bool MRT>
cudaError_t launch_step_w(const DomDesc& d, const DomDesc* d_descs, const WorkItem* d_items,
                          int n_items, int n_dom, int parity, int bx, int rows, int band_mul, int grid_p,
                          int* sched, bool one_body, cudaStream_t s)
{
    if (one_body && !(n_dom == 1 && d_items == nullptr))
        return launch_step_t<Real, MRT, 0>(d, d_descs, d_items, n_items, n_dom, parity, bx, rows,
                                           band_mul, grid_p, sched, s);
    switch (bx) {
        case 64:
            return launch_step_t<Real, MRT, 2>(d, d_descs, d_items, n_items, n_dom, parity, bx,
                                               rows, band_mul, grid_p, sched, s);
        case 128:
            return launch_step_t<Real, MRT, 4>(d, d_descs, d_items, n_items, n_dom, parity, bx,
                                               rows, band_mul, grid_p, sched, s);
        case 256:
            return launch_step_t<Real, MRT, 8>(d, d_descs, d_items, n_items, n_dom, parity, bx,
                                               rows, band_mul, grid_p, sched, s);
        default:
            return launch_step_t<Real, MRT, 0>(d, d_descs, d_items, n_items, n_dom, parity, bx,
                                               rows, band_mul, grid_p, sched, s);
    }
}

template <typename Real>
int launch_step_prec(int coll, const DomDesc& d, const DomDesc* d_descs, const WorkItem* d_items,
                     int n_items, int n_dom, int parity, int bx, int rows, int band_mul, int grid_p,
                     int* sched, bool one_body, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    return int(coll ? launch_step_w<Real, true>(d, d_descs, d_items, n_items, n_dom, parity, bx,
                                                rows, band_mul, grid_p, sched, one_body, s)
                    : launch_step_w<Real, false>(d, d_descs, d_items, n_items, n_dom, parity, bx,
                                                 rows, band_mul, grid_p, sched, one_body, s));
}

// Resident CTAs per SM of the batched kernels (single: of the single-domain
// kernels) for a launch shape (0 on error).
template <bool MRT, int NWC>
int batch_occupancy_compact_t(int bx, bool single)
{
    int n = 0;
    const size_t smem = StageLayoutC(bx / 32, kStagesC).total();
    const cudaError_t e =
        single ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     &n, step_single_compact_kernel<MRT, NWC>, bx + 32, smem)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     &n, step_batch_compact_kernel<MRT, NWC>, bx + 32, smem);
    return e == cudaSuccess ? n : 0;
}

template <typename Real, bool MRT, int NWC>
int batch_occupancy_t(int bx, bool single)
{
    int n = 0;
    const size_t smem = StageLayout<Real>(bx / 32, kStages<Real>).total();
    const cudaError_t e =
        single ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     &n, step_single_kernel<Real, MRT, NWC>, bx + 32, smem)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                     &n, step_batch_kernel<Real, MRT, NWC>, bx + 32, smem);
    return e == cudaSuccess ? n : 0;
}

template <bool MRT>
int batch_occupancy_compact_w(int bx, bool single)
{
    switch (bx) {
        case 32: return batch_occupancy_compact_t<MRT, 1>(bx, single);
        case 64: return batch_occupancy_compact_t<MRT, 2>(bx, single);
        case 96: return batch_occupancy_compact_t<MRT, 3>(bx, single);
        case 128: return batch_occupancy_compact_t<MRT, 4>(bx, single);
        case 256: return batch_occupancy_compact_t<MRT, 8>(bx, single);
        default: return batch_occupancy_compact_t<MRT, 0>(bx, single);
    }
}

template <typename Real, bool MRT>
int batch_occupancy_w(int bx, bool single)
{
    switch (bx) {
        case 64: return batch_occupancy_t<Real, MRT, 2>(bx, single);
        case 128: return batch_occupancy_t<Real, MRT, 4>(bx, single);
        case 256: return batch_occupancy_t<Real, MRT, 8>(bx, single);
        default: return batch_occupancy_t<Real, MRT, 0>(bx, single);
    }
}

template <bool MRT, int NWC>
cudaError_t allow_large_smem_compact()
{
    const int bytes = 200 * 1024;
    cudaError_t e = cudaFuncSetAttribute(step_single_compact_kernel<MRT, NWC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_batch_compact_kernel<MRT, NWC>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    // the classes of a batch run side by side: one carveout for all of them
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_batch_compact_kernel<MRT, NWC>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

// Opt every instantiation in to large dynamic shared memory.
template <typename Real, bool MRT, int NWC>
cudaError_t allow_large_smem_one()
{
    const int bytes = 200 * 1024;
    cudaError_t e = cudaFuncSetAttribute(step_single_kernel<Real, MRT, NWC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_batch_kernel<Real, MRT, NWC>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

template <typename Real>
int prepare_step_prec()
{
    cudaError_t e = cudaSuccess;
    const cudaError_t r[] = {
        allow_large_smem_one<Real, false, 0>(), allow_large_smem_one<Real, false, 2>(),
        allow_large_smem_one<Real, false, 4>(), allow_large_smem_one<Real, false, 8>(),
        allow_large_smem_one<Real, true, 0>(),  allow_large_smem_one<Real, true, 2>(),
        allow_large_smem_one<Real, true, 4>(),  allow_large_smem_one<Real, true, 8>()};
    for (cudaError_t v : r)
        if (v != cudaSuccess) e = v;
    return int(e);
}

}  // namespace lbfe
