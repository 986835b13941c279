// FP32 instantiation of the fused step kernels (see lb_step_kernels.cuh).
#include "lb_step_kernels.cuh"

namespace lbfe {

int launch_step_f32(int coll, const DomDesc& d, const DomDesc* d_descs, const WorkItem* d_items,
                    int n_items, int n_dom, int parity, int bx, int rows, int band_mul, int grid_p,
                    int* sched, bool one_body, void* stream)
{
    if (d.compact) {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        return int(coll ? launch_step_compact_w<true>(d, d_descs, d_items, n_items, n_dom, parity,
                                                      bx, rows, band_mul, grid_p, sched, one_body, s)
                        : launch_step_compact_w<false>(d, d_descs, d_items, n_items, n_dom,
                                                       parity, bx, rows, band_mul, grid_p, sched,
                                                       one_body, s));
    }
    return launch_step_prec<float>(coll, d, d_descs, d_items, n_items, n_dom, parity, bx, rows,
                                   band_mul, grid_p, sched, one_body, stream);
}

int batch_occupancy_f32(int coll, int compact, int bx, int single)
{
    if (compact)
        return coll ? batch_occupancy_compact_w<true>(bx, single != 0)
                    : batch_occupancy_compact_w<false>(bx, single != 0);
    return coll ? batch_occupancy_w<float, true>(bx, single != 0)
                : batch_occupancy_w<float, false>(bx, single != 0);
}

int prepare_step_f32()
{
    int e = prepare_step_prec<float>();
    const cudaError_t r[] = {
        allow_large_smem_compact<false, 0>(), allow_large_smem_compact<false, 1>(),
        allow_large_smem_compact<false, 2>(), allow_large_smem_compact<false, 3>(), allow_large_smem_compact<false, 4>(),
        allow_large_smem_compact<false, 8>(), allow_large_smem_compact<true, 0>(),
        allow_large_smem_compact<true, 1>(),  allow_large_smem_compact<true, 2>(),  allow_large_smem_compact<true, 3>(),
        allow_large_smem_compact<true, 4>(),  allow_large_smem_compact<true, 8>()};
    for (cudaError_t v : r)
        if (v != cudaSuccess) e = int(v);
    return e;
}

}  // namespace lbfe
