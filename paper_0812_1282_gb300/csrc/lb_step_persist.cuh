// Persistent multi-step form of the batched compact step, in its own
// translation unit (lb_step_persist.cu).
#pragma once

#include "lb_step_kernels.cuh"

namespace lbfe {

// Persistent multi-step form of the batched compact kernel: one launch runs
// n_steps time steps of one schedule class.  The producer warp takes
// tickets t = s n_items + i (work item i of step s; every ticket of step s
// before any of step s + 1) from the device counter sched[0].  Before it
// copies item i's rows for step s it waits until each item that step reads
// from (i itself and the row blocks and strips within reach of its halo:
// dep_idx[dep_off[i] .. dep_off[i + 1])) has finished step s - 1, which also
// means they are done reading the rows item i now overwrites.  The compute
// warps publish an item's step in flags[i] (steps done in this launch)
// once all its rows are stored.  A CTA takes a ticket only while it runs and
// tickets go out in order, so the oldest ticket in flight never waits: the
// waits end however many CTAs are resident, and each is also bounded in
// time (a give-up sets *err and the CTA stops taking tickets).  Step s
// reads buffer parity0 ^ (s & flip).  The last CTA to finish resets the
// counters and the flags for the next launch.
template <bool MRT, int NWC>
__global__ void __maxnreg__(96)
    step_persist_compact_kernel(const DomDesc* __restrict__ descs,
                                const WorkItem* __restrict__ items,
                                const int* __restrict__ dep_off, const int* __restrict__ dep_idx,
                                int n_items, int n_steps, int parity0, int flip, int* flags,
                                int* sched, unsigned* err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int tags[kStagesC];
    __shared__ NodeParams<float> tile_prm;
    __shared__ DomDesc tile_desc;
    __shared__ int last_cta;
    constexpr int S = kStagesC;
    const int NW = NWC > 0 ? NWC : int(blockDim.x >> 5) - 1;
    init_stages_c<S>(smem, NW);
    const int warp = int(threadIdx.x >> 5), lane = int(threadIdx.x & 31);
    const int n_tickets = n_items * n_steps;
    unsigned q = 0;
    if (warp == 0) {
        int t = 0;
        if (lane == 0) t = atomicAdd(sched, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        for (;;) {
            if (t >= n_tickets) {
                produce_end<float, S, NWC>(smem, NW, q, tags, err);
                break;
            }
            int tn = 0;  // the next ticket, fetched while this one is produced
            if (lane == 0) tn = atomicAdd(sched, 1);
            const int s = t / n_items, it = t - s * n_items;
            const WorkItem w = items[it];
            bool ok = true;
            if (s > 0) {
                const int k1 = dep_off[it + 1];
                for (int k = dep_off[it]; k < k1 && ok; ++k) ok = flag_wait(flags + dep_idx[k], s, err);
                // one decision for the warp (a lane's wait may give up alone)
                ok = __all_sync(0xffffffffu, ok);
            }
            fence_proxy_async_global();
            const DomDesc D = descs[w.dom];
            produce_tile_c<S, NWC>(D, parity0 ^ (s & flip), w.x0, w.y0, w.rows, w.cols, smem, NW,
                                   q, tags, t);
            t = ok ? __shfl_sync(0xffffffffu, tn, 0) : n_tickets;
        }
        drain_stages<float, S, NWC>(smem, NW, q, err);
    } else {
        for (;;) {
            const int t = next_tag<float, S, NWC>(smem, NW, q, tags, err);
            if (named_sync_or(kComputeBarrier, 32 * NW, t < 0 || t >= n_tickets)) break;
            const int s = t / n_items, it = t - s * n_items;
            const WorkItem w = items[it];
            if (warp == 1 && lane == 0) {
                tile_desc = descs[w.dom];
                tile_prm = node_params<float>(tile_desc);
            }
            named_sync(kComputeBarrier, 32 * NW);
            consume_tile_c<MRT, S, NWC, true>(tile_desc, parity0 ^ (s & flip), w.x0, w.y0, w.rows,
                                              w.cols, smem, NW, warp - 1, q, &tile_prm,
                                              (w.flags & kItemSeal) != 0);
            // every row of the item is stored: publish its step
            fence_proxy_async_global();
            named_sync(kComputeBarrier, 32 * NW);
            if (warp == 1 && lane == 0) {
                __threadfence();
                st_release_gpu(flags + it, s + 1);
            }
        }
    }
    // the whole CTA is done and its flags are out: count it; the last CTA
    // resets the counters and the flags
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last_cta = atomicAdd(sched + 1, 1) == int(gridDim.x) - 1;
    }
    __syncthreads();
    if (last_cta) {
        __threadfence();
        for (int k = int(threadIdx.x); k < n_items; k += int(blockDim.x)) flags[k] = 0;
        if (threadIdx.x == 0) {
            sched[0] = 0;
            sched[1] = 0;
        }
        __threadfence();
    }
}

template <bool MRT, int NWC>
cudaError_t launch_persist_compact_t(const PersistLaunch& a, cudaStream_t s)
{
    const size_t smem = StageLayoutC(a.bx / 32, kStagesC).total();
    step_persist_compact_kernel<MRT, NWC><<<a.grid, a.bx + 32, smem, s>>>(
        a.descs, a.items, a.dep_off, a.dep_idx, a.n_items, a.n_steps, a.parity0, a.flip, a.flags,
        a.sched, a.err);
    return cudaGetLastError();
}

template <bool MRT>
cudaError_t launch_persist_compact_w(const PersistLaunch& a, cudaStream_t s)
{
    switch (a.bx) {
        case 32: return launch_persist_compact_t<MRT, 1>(a, s);
        case 64: return launch_persist_compact_t<MRT, 2>(a, s);
        case 96: return launch_persist_compact_t<MRT, 3>(a, s);
        case 128: return launch_persist_compact_t<MRT, 4>(a, s);
        case 256: return launch_persist_compact_t<MRT, 8>(a, s);
        default: return launch_persist_compact_t<MRT, 0>(a, s);
    }
}

template <bool MRT, int NWC>
int persist_occupancy_t(int bx)
{
    int n = 0;
    const size_t smem = StageLayoutC(bx / 32, kStagesC).total();
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_persist_compact_kernel<MRT, NWC>,
                                                      bx + 32, smem) != cudaSuccess)
        return 0;
    return n;
}

// Registers per thread and shared memory per CTA (static + dynamic) of the
// persistent kernel for a launch shape (false on error).
template <bool MRT, int NWC>
bool persist_footprint_t(int bx, int* regs, size_t* smem)
{
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, step_persist_compact_kernel<MRT, NWC>) != cudaSuccess) return false;
    *regs = fa.numRegs;
    *smem = fa.sharedSizeBytes + StageLayoutC(bx / 32, kStagesC).total();
    return true;
}

template <bool MRT>
bool persist_footprint_w(int bx, int* regs, size_t* smem)
{
    switch (bx) {
        case 32: return persist_footprint_t<MRT, 1>(bx, regs, smem);
        case 64: return persist_footprint_t<MRT, 2>(bx, regs, smem);
        case 96: return persist_footprint_t<MRT, 3>(bx, regs, smem);
        case 128: return persist_footprint_t<MRT, 4>(bx, regs, smem);
        case 256: return persist_footprint_t<MRT, 8>(bx, regs, smem);
        default: return persist_footprint_t<MRT, 0>(bx, regs, smem);
    }
}

template <bool MRT>
int persist_occupancy_w(int bx)
{
    switch (bx) {
        case 32: return persist_occupancy_t<MRT, 1>(bx);
        case 64: return persist_occupancy_t<MRT, 2>(bx);
        case 96: return persist_occupancy_t<MRT, 3>(bx);
        case 128: return persist_occupancy_t<MRT, 4>(bx);
        case 256: return persist_occupancy_t<MRT, 8>(bx);
        default: return persist_occupancy_t<MRT, 0>(bx);
    }
}

// Large dynamic shared memory, and the largest shared-memory carveout: the
// classes of a persistent schedule run side by side for a whole launch, and
// CTAs of kernels that asked for different carveouts could not share an SM.
template <bool MRT, int NWC>
cudaError_t allow_large_smem_persist()
{
    cudaError_t e = cudaFuncSetAttribute(step_persist_compact_kernel<MRT, NWC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(step_persist_compact_kernel<MRT, NWC>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

}  // namespace lbfe
