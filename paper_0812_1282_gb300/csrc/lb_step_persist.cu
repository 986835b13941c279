// Persistent multi-step batched compact kernel (see lb_step_persist.cuh),
// in a translation unit of its own so that it compiles beside the others.
#include "lb_step_persist.cuh"

namespace lbfe {

int launch_persist(int coll, const PersistLaunch& a, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (a.n_items <= 0 || a.n_steps <= 0 || a.grid <= 0) return int(cudaErrorInvalidValue);
    return int(coll ? launch_persist_compact_w<true>(a, s) : launch_persist_compact_w<false>(a, s));
}

int persist_occupancy(int coll, int block_x)
{
    return coll ? persist_occupancy_w<true>(block_x) : persist_occupancy_w<false>(block_x);
}

int persist_footprint(int coll, int block_x, int* regs, size_t* smem)
{
    const bool ok = coll ? persist_footprint_w<true>(block_x, regs, smem)
                         : persist_footprint_w<false>(block_x, regs, smem);
    return ok ? 0 : int(cudaErrorInvalidValue);
}

int prepare_persist()
{
    int e = 0;
    const cudaError_t r[] = {
        allow_large_smem_persist<false, 0>(), allow_large_smem_persist<false, 1>(),
        allow_large_smem_persist<false, 2>(), allow_large_smem_persist<false, 3>(),
        allow_large_smem_persist<false, 4>(), allow_large_smem_persist<false, 8>(),
        allow_large_smem_persist<true, 0>(),  allow_large_smem_persist<true, 1>(),
        allow_large_smem_persist<true, 2>(),  allow_large_smem_persist<true, 3>(),
        allow_large_smem_persist<true, 4>(),  allow_large_smem_persist<true, 8>()};
    for (cudaError_t v : r)
        if (v != cudaSuccess) e = int(v);
    return e;
}

}  // namespace lbfe
