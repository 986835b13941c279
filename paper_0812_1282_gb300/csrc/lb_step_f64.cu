// FP64 instantiation of the fused step kernels (see lb_step_kernels.cuh).
#include "lb_step_kernels.cuh"

namespace lbfe {

int launch_step_f64(int coll, const DomDesc& d, const DomDesc* d_descs, const WorkItem* d_items,
                    int n_items, int n_dom, int parity, int bx, int rows, int band_mul, int grid_p,
                    int* sched, bool one_body, void* stream)
{
    return launch_step_prec<double>(coll, d, d_descs, d_items, n_items, n_dom, parity, bx, rows,
                                    band_mul, grid_p, sched, one_body, stream);
}

int batch_occupancy_f64(int coll, int bx, int single)
{
    return coll ? batch_occupancy_w<double, true>(bx, single != 0)
                : batch_occupancy_w<double, false>(bx, single != 0);
}

int prepare_step_f64() { return prepare_step_prec<double>(); }

}  // namespace lbfe
