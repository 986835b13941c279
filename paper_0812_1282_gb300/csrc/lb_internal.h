// Internal host/device interface of the library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace lbfe {

// Row layout: logical column x of a row lives at physical column x + kXOff;
// physical columns kXOff-2, kXOff-1 hold copies of logical nx-2, nx-1 and
// physical nx+kXOff, nx+kXOff+1 copies of logical 0, 1 (periodic ghosts,
// kept current by every kernel that writes populations).  pitch >= nx + 8.
constexpr int kXOff = 4;

// Node columns of one strip of the compact step (FP32, compact g storage)
// for a CTA of bx = 32 NW compute threads: each compute warp covers 62 new
// columns, less the halo the phi stencil needs, rounded down to a multiple
// of 4 so that strips start on 16-byte boundaries.
__host__ __device__ constexpr int compact_strip(int bx) { return (62 * (bx / 32) - 2) / 4 * 4; }

// One domain as the kernels see it.  Populations live in two ping-pong
// buffers; buffer b holds f at f[b] and g at g[b], each 9 planes of
// `plane` elements (pitch * ny, x fastest).
struct DomDesc {
    void* f[2];
    void* g[2];
    long long plane;   // elements per population plane
    int nx, ny, pitch;
    int walls;         // 1: bounce-back walls below row 0 and above row ny-1
    int step2;         // zero equilibrium velocity on wall rows (Sec. V, Step 2)
    int step2_relax_j; // MRT: relax wall-row momentum at rate 1 (alternative reading)
    int compact;       // FP32, tau_phi = 1: g stored as (phi word, Gamma mu, u_eq) in
                       // g planes 0..3 (lb_step_compact.cuh)
    int wet_k;         // wetting ghost: phi(ghost) = phi(k - 1 rows inside) - k h, with
                       // k = 2 (mirror about the boundary row) or 1 (one-sided across
                       // the wall plane); at obstacles mean phi(s + k d) - k h
    double a, kappa, gamma;   // free energy and mobility parameters
    double omega_phi;         // 1 / tau_phi
    double tau_c0, tau_c1;    // tau_rho(phi) = tau_c0 + tau_c1 * phi  (Eq. tau)
    double h_bot, h_top;      // wetting gradients
    // lookup table of Sec. V (lut_kmax = 0: exact tau): tau = lut_lo + k lut_step,
    // k = nearest integer to (tau - lut_lo) lut_inv, clamped to [0, lut_kmax]
    double lut_lo, lut_step, lut_inv, lut_kmax;
    unsigned* err;            // device error word (bounded waits that gave up)
    // the same parameters rounded to float once on the host (the FP32 step
    // reads these; converting in the kernel would run on the slow FP64 pipe)
    float fa, fkappa, fgamma, fomega_phi, ftau_c0, ftau_c1, fh_bot, fh_top;
    float flut_lo, flut_step, flut_inv, flut_kmax;
    // Obstacles (nullptr: none).  cls[y * nx + x] = 0 for a fluid node, k in
    // 1..kMaxClass for a solid node of wetting class k with inward-normal
    // wetting gradient hcls[k].
    const unsigned char* cls;
    double hcls[8];
    float fhcls[8];
};

constexpr int kMaxClass = 7;
// Class of a node-bounce-back wall node (rows 0 and ny - 1 of a walled
// domain; the wetting gradient is the wall's h_bot / h_top).
constexpr int kNodeWall = 8;

// A rectangular piece of one domain processed by one CTA: columns
// [x0, x0 + cols) and rows [y0, y0 + rows).  cols = 0 means the kernel's
// full strip width (clipped to the domain).
struct WorkItem {
    int dom, x0, y0, rows, cols;
    int flags;  // kItemSeal: a whole-domain strip completes its rows' edge sectors
};
constexpr int kItemSeal = 1;

// Per-domain reduction result written by the moments kernels.
struct StatsOut {
    double mass, order, mom_x, mom_y, max_u;
    double nonfinite;
};

constexpr int kStatsFields = 6;

// Launchers implemented in the .cu files.  All return a cudaError_t value
// cast to int (0 = success) and enqueue on `stream`.
// sched: two device ints, zero between launches (batched form only).
// band_mul: single-domain form, the order in which row bands start (grid
// row g takes band g band_mul mod the band count; 1 = in order).
// one_body: batched form, launch the kernel built for any block width (the
// warp count read from the block size) rather than the one built for this
// width, so that the classes of a schedule, which run side by side, share
// one code body in the SMs' instruction caches.
int launch_step(int precision, int coll, const DomDesc& d, const DomDesc* d_descs,
                const WorkItem* d_items, int n_items, int n_dom, int parity, int block_x,
                int rows, int band_mul, int grid_persistent, int* sched, bool one_body,
                void* stream);

// One launch of the persistent multi-step batched compact kernel (FP32,
// compact g storage) over one schedule class: items, dep_off (n_items + 1
// entries) and flags are the class's slices; dep_idx holds class-local item
// indices.
struct PersistLaunch {
    const DomDesc* descs;
    const WorkItem* items;
    const int* dep_off;
    const int* dep_idx;
    int* flags;
    int* sched;
    unsigned* err;
    int n_items, n_steps, parity0, flip, bx, grid;
};
int launch_persist(int coll, const PersistLaunch& a, void* stream);
// Resident CTAs per SM of the persistent kernel (0 on error), and its
// shared-memory opt-in (once per device, outside any capture).
int persist_occupancy(int coll, int block_x);
int persist_footprint(int coll, int block_x, int* regs, size_t* smem);
int prepare_persist();

int launch_init_phi_drop(int precision, const DomDesc& d, double* phi0, double R, double cx,
                         double cy, void* stream);
int launch_init_phi_random(int precision, const DomDesc& d, double* phi0, double amp,
                           unsigned long long seed, void* stream);
int launch_init_eq(int precision, const DomDesc& d, const double* phi0, int parity,
                   void* stream);
// phi0 rows (nx per row, contiguous, device-addressable) into the pitched field.
int launch_copy_rows(const DomDesc& d, const double* src, double* phi0, void* stream);
int launch_moments(int precision, const DomDesc& d, int parity, int row0, int nrows,
                   double* rho, double* phi, double* ux, double* uy, long long ld,
                   double* partials, int max_partials, StatsOut* out, void* stream);
int launch_crossings(int precision, const DomDesc& d, int parity, double* pts, int* count,
                     int cap, void* stream);
int launch_fill_ghosts(int precision, const DomDesc& d, int parity, void* stream);

// Domains with obstacles (d.cls != nullptr): one time step (one kernel),
// the initial equilibrium, and the rest state of the solid nodes of buffer b.
int launch_geo_step(int precision, int coll, const DomDesc& d, int parity, void* stream);
int launch_geo_init_eq(int precision, const DomDesc& d, const double* phi0, int parity,
                       void* stream);
int launch_geo_solid_rest(int precision, const DomDesc& d, int b, void* stream);

// Opt the step kernels in to large dynamic shared memory (call once per
// device before the first launch, outside any stream capture).
int prepare_step_kernels();

// Per-precision halves of launch_step / prepare_step_kernels.
int launch_step_f32(int coll, const DomDesc& d, const DomDesc* d_descs, const WorkItem* d_items,
                    int n_items, int n_dom, int parity, int bx, int rows, int band_mul, int grid_p,
                    int* sched, bool one_body, void* stream);
int launch_step_f64(int coll, const DomDesc& d, const DomDesc* d_descs, const WorkItem* d_items,
                    int n_items, int n_dom, int parity, int bx, int rows, int band_mul, int grid_p,
                    int* sched, bool one_body, void* stream);
int prepare_step_f32();
int prepare_step_f64();

// Resident CTAs per SM of the batched (single-domain) step kernel for a
// launch shape (0 if the shape is not supported or the query fails).
int step_batch_occupancy(int precision, int coll, int compact, int block_x);
int step_single_occupancy(int precision, int coll, int compact, int block_x);
int batch_occupancy_f32(int coll, int compact, int bx, int single);
int batch_occupancy_f64(int coll, int bx, int single);

// Dynamic shared memory of the step kernel for a block width (0 if the
// width is not supported for this precision).
size_t step_smem_bytes(int precision, int block_x);

int max_partials_needed(int nx, int ny);

// Launch the bounded-wait self-check and return the error word it left.
int run_wait_selfcheck(void* stream, unsigned* word);

}  // namespace lbfe
