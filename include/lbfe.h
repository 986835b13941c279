/*
 * lbfe.h -- C ABI of the GB300 (sm_103a) free-energy binary-fluid lattice
 * Boltzmann library.
 *
 * The method is the D2Q9 binary-fluid scheme of Pooley, Kusumaatmaja &
 * Yeomans, "Contact line dynamics in binary lattice Boltzmann simulations"
 * (arXiv:0812.1282): a density distribution f_i and an order-parameter
 * distribution g_i (Sec. III.A, Eq. moments), the Landau free energy of
 * Sec. II (Eqs. freeen, bulkfe, chempot, pressten, p0), the equilibria and
 * isotropic stencils of Appendix A (Eqs. equilibrium, feq0, best), BGK
 * (Eqs. latbolt, gevo) or multiple-relaxation-time collision (Eqs. mrtlb,
 * Matrix, diag) with the phi-dependent relaxation time of Eq. (tau), mid-link
 * bounce-back walls carrying the wetting gradient d(phi)/dn (Sec. II, IV),
 * and the four-step algorithm of Sec. V.
 *
 * Conventions shared by every entry point
 *  - Lattice units: c = dx = dt = 1.  Velocity order e0=(0,0) e1=(1,0)
 *    e2=(-1,0) e3=(0,1) e4=(0,-1) e5=(1,1) e6=(-1,-1) e7=(-1,1) e8=(1,-1).
 *  - A domain is nx columns by ny rows (nx, ny >= 3).  x is periodic.  y is
 *    periodic (walls = 0) or closed by mid-link bounce-back walls half a
 *    spacing below row 0 and above row ny-1 (walls = 1).
 *  - Host field arrays are row-major [ny][nx] doubles (x fastest);
 *    population arrays are [9][ny][nx] doubles.
 *  - The stored state after n steps is the post-collision population set
 *    of step n; observables (rho, phi, u) are its moments (Eq. moments).
 *    rho and phi equal those of the pre-collision state exactly in exact
 *    arithmetic; so does rho*u except at Step-2 boundary nodes under BGK.
 *  - Every call returns LB_OK (0) or a negative LB_ERR_* code and never
 *    aborts the process; lb_last_error() gives a message for the calling
 *    thread.  Work is enqueued on the handle's CUDA stream; calls that
 *    return data to the host synchronise that stream first.
 *  - The library never falls back to the CPU: without a usable CUDA device
 *    lb_create returns LB_ERR_CUDA.
 */
#ifndef LBFE_H
#define LBFE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LB_OK 0
#define LB_ERR_INVALID_ARG (-1) /* bad size, parameter, index or buffer      */
#define LB_ERR_CUDA (-2)        /* a CUDA runtime call failed                */
#define LB_ERR_NONFINITE (-3)   /* NaN/Inf found in the state                 */
#define LB_ERR_TIMEOUT (-4)     /* a bounded device wait gave up              */
#define LB_ERR_NO_INTERFACE (-5) /* fewer than 3 interface points to fit      */
#define LB_ERR_CAPACITY (-6)    /* interface-point buffer too small           */

#define LB_BGK 0 /* single relaxation time, Eq. (latbolt)                   */
#define LB_MRT 1 /* multiple relaxation time, Eqs. (mrtlb), (Matrix), (diag) */

#define LB_FP32 0 /* populations stored in FP32 as deviations from the rest
                     state (rho = 1, u = 0, phi = 0); arithmetic in FP32 */
#define LB_FP64 1 /* populations and arithmetic in FP64 */

typedef struct lb_params {
    double a;          /* bulk free-energy constant, psi = a(-phi^2/2 + phi^4/4), Eq. (bulkfe) */
    double kappa;      /* gradient-energy constant, Eq. (freeen)                         */
    double gamma_mob;  /* Gamma of the g equilibrium, Eq. (Mobility), Appendix A          */
    double tau_phi;    /* relaxation time of g, Eq. (gevo); Sec. III.B sets 1 under MRT   */
    double tau_alpha;  /* tau_rho in the phi = +1 phase, Eq. (tau)                        */
    double tau_beta;   /* tau_rho in the phi = -1 phase, Eq. (tau)                        */
    double h_bottom;   /* wetting gradient: inward-normal d(phi)/dn at the y = -1/2 wall, */
    double h_top;      /*   and at the y = ny - 1/2 wall (xi = kappa h, Sec. II)          */
    int collision;       /* LB_BGK or LB_MRT                                              */
    int zero_u_at_walls; /* Step 2 of Sec. V: equilibrium velocity 0 on wall rows          */
    int precision;       /* LB_FP32 or LB_FP64                                            */
    int walls;           /* 1: bounce-back walls in y; 0: periodic y                      */
    int step2_relax_momentum; /* MRT only: on Step-2 rows the momentum rows of Eq. (diag)
                                 relax at rate 1 (wall-row momentum set to zero) instead of
                                 the literal rate 0 of the conserved moments (default 0) */
    int mrt_lut;         /* MRT only: 0 (default) uses the exact tau(phi) of Eq. (tau) at
                            every node; n >= 2 uses the nearest of n viscosities spaced
                            evenly between tau_beta and tau_alpha (ends included, the end
                            values beyond them): the lookup table of Sec. V            */
    int compact_g;       /* 1: store g compactly (FP32 and tau_phi = 1 only; no obstacles).
                            With tau_phi = 1 the post-collision g of a node is its
                            equilibrium (Eq. gevo), fixed by phi, Gamma mu and u_eq, so the
                            state keeps those four numbers instead of nine g values:
                            104 instead of 144 bytes of traffic per node update.  The
                            scheme is the same; g'_0 = phi - sum g'_i is implicit.
                            lb_set_populations is not available on such a handle.
                            Default 0. */
    int wetting_rule;    /* discretisation of the wetting condition of Sec. II (the
                            inward normal derivative of phi at a wall equals h): 0
                            (default) mirrors phi about the boundary row, ghost
                            phi(x,-1) = phi(x,1) - 2 h, so the isotropic gradient of the
                            boundary row is h; 1 takes the one-sided difference across
                            the wall plane, phi(x,-1) = phi(x,0) - h.  At obstacles the
                            same rule along each direction towards the fluid
                            (phi(s) = mean phi(s + 2d) - 2h, or mean phi(s + d) - h). */
} lb_params;

/* Diagnostics of one domain (sums over all nodes, in FP64). */
typedef struct lb_stats {
    double mass;      /* sum rho                        */
    double order;     /* sum phi                        */
    double mom_x;     /* sum rho u_x                    */
    double mom_y;     /* sum rho u_y                    */
    double max_u;     /* max |u|  (spurious-current norm, Sec. IV) */
    long long nonfinite; /* number of nodes whose moments are not finite */
    long long step;      /* steps taken since the last initialisation  */
} lb_stats;

typedef struct lb_handle lb_handle;

/* Device bytes a handle needs for n_dom domains of the given sizes and
 * precision (state ping-pong buffers plus workspace).  Returns 0 on invalid
 * arguments. */
size_t lb_device_bytes(int precision, int n_dom, const int* nx, const int* ny);

/* Create one domain (a batch of one).
 *  stream:   cudaStream_t the handle enqueues on (NULL: the legacy default
 *            stream).  The caller keeps it alive while the handle lives.
 *  dev_mem:  optional caller-owned device buffer of at least
 *            lb_device_bytes(...) bytes, 256-byte aligned (e.g. a PyTorch
 *            tensor); NULL makes the library cudaMalloc and own it.
 * Errors: LB_ERR_INVALID_ARG for nx or ny < 3, non-positive a, kappa or
 * gamma_mob, tau_phi <= 1/2, a tau_rho(phi) <= 1/2 anywhere on
 * phi in [-1.1, 1.1], a domain whose 9 planes exceed 2^31 elements, or a
 * too-small dev_mem; LB_ERR_CUDA when no device is usable. */
int lb_create(const lb_params* p, int nx, int ny, void* stream, void* dev_mem,
              size_t dev_bytes, lb_handle** out);

/* Create n_dom independent domains that advance together (one launch per
 * step over all of them).  per_dom[d], nx[d], ny[d] describe domain d;
 * precision and collision must be the same for all domains.  Other rules
 * as lb_create. */
int lb_create_batch(const lb_params* per_dom, const int* nx, const int* ny, int n_dom,
                    void* stream, void* dev_mem, size_t dev_bytes, lb_handle** out);

/* Release the handle (and the device memory it allocated itself). */
void lb_destroy(lb_handle* h);

/* Initial state of domain dom: phi0 given by one of the initialisers below,
 * rho = 1, u = 0, and f = f^eq, g = g^eq of that state (Appendix A, with the
 * stencils and wetting ghost rows of the domain).  Resets the step count. */

/* Drop of radius R centred at (cx, cy): phi0 = tanh((R - d)/l), l =
 * sqrt(2 kappa / a) (the flat-interface profile of Eq. chempot; width
 * W = 2l, Sec. IV).  cy = -0.5 puts the centre on the bottom wall plane. */
int lb_init_drop(lb_handle* h, int dom, double R, double cx, double cy);

/* Spinodal start: phi0 uniform in [-amp, amp), node (x, y) taking draw
 * k = y*nx + x of the SplitMix64 stream seeded with `seed`
 * (mix(seed + (k+1) * 0x9E3779B97F4A7C15), top 53 bits). */
int lb_init_random(lb_handle* h, int dom, double amp, unsigned long long seed);

/* Arbitrary phi0: host (on_device = 0) or device (1) array [ny][nx] of
 * doubles, read before the call returns.  A page-locked host array is read
 * by a kernel through its device address; pageable host memory is copied. */
int lb_init_phi(lb_handle* h, int dom, const double* phi0, int on_device);

/* Advance every domain of the handle by n >= 0 time steps (Steps 1-4 of
 * Sec. V, pull form).  Asynchronous on the handle's stream; repeated step
 * blocks are replayed from captured CUDA graphs. */
int lb_step(lb_handle* h, int n);

/* Moments of domain dom.  rho, phi, ux, uy: [ny][nx] double buffers on the
 * host (on_device = 0) or the device (1); any may be NULL.  When every
 * requested host buffer is page-locked the kernel writes them directly;
 * otherwise they are filled through a device staging buffer.  stats may be
 * NULL.  Synchronises the stream.  Returns LB_ERR_NONFINITE (after filling
 * the outputs) if a node's moments are not finite. */
int lb_moments(lb_handle* h, int dom, int on_device, double* rho, double* phi,
               double* ux, double* uy, lb_stats* stats);

/* Contact angle of a drop sitting on the bottom wall of domain dom (Sec. IV,
 * Fig. 1): every horizontal and vertical link whose ends have phi > 0 and
 * phi < 0 gives a phi = 0 point by linear interpolation; points closer than
 * `exclude` to the wall plane y = -1/2 are dropped; a least-squares circle
 * (algebraic start, geometric Gauss-Newton refinement) gives
 * theta = 90 + asin((yc + 1/2)/R) degrees, measured through phi > 0.
 * Any output pointer may be NULL.  LB_ERR_NO_INTERFACE if fewer than 3
 * points remain, LB_ERR_CAPACITY if the interface is too long for the
 * point buffer (16 (nx + ny) points). */
int lb_contact_angle(lb_handle* h, int dom, double exclude, double* theta_deg,
                     double* R, double* xc, double* yc);

/* Solid obstacles in domain dom (the capillary geometry of Sec. VI; the
 * paper states bounce-back and the wetting condition for flat walls only,
 * and they are read here node by node).
 *  cls:     host array [ny][nx]; 0 marks a fluid node, k in 1..7 a solid node
 *           of wetting class k, 8 a node-bounce-back wall node (below).
 *           NULL removes the obstacles.  Copied before the call returns.
 *  h_class: n_class (1..8) inward-normal wetting gradients, h_class[k] for
 *           class k (entry 0 unused).
 * Rules: a pull from a solid node is bounced back (mid-link, as at a wall);
 * Step 2 acts on fluid nodes with a solid neighbour; a solid node next to
 * fluid takes the ghost value mean_d phi(s + 2d) - 2 h over the axis
 * directions d with a fluid neighbour s + d (the flat-wall mirror; the
 * diagonal directions if s touches fluid only through a corner).  Walls
 * (params.walls) stay solid rows with h_bottom / h_top.  Solid nodes hold
 * the rest state and report rho = phi = u = 0; they are left out of the
 * statistics and of the interface points.  A domain with obstacles is
 * stepped by one plain kernel per step instead of the staged one.
 * Node bounce-back (Fig. 4b, the wall lying on the boundary nodes; the
 * paper gives no more detail): class 8 in row 0 or row ny - 1 of a walled
 * domain of at least 4 rows, read as the full-way scheme.  A wall node
 * streams like a fluid node (its pulls from beyond the domain bounce back)
 * and reverses every population instead of colliding; its fluid neighbours
 * see phi(x, 0) = phi(x, 1) - h_bottom (phi(x, ny - 1) = phi(x, ny - 2) -
 * h_top) and are Step-2 nodes; it reports no moments of its own and is
 * initialised to the rest equilibrium of that phi value.  The no-slip planes
 * then lie half a spacing inside the wall-node rows.
 * The state must be initialised again afterwards (lb_init_*).
 * Errors: LB_ERR_INVALID_ARG for a class out of range or without a
 * gradient, a non-finite gradient, a map without fluid, a solid node whose
 * mirror node s + 2d is solid or a wall node (features thinner than two
 * nodes), or a wall node outside the outer rows of a walled domain of at
 * least 4 rows or without fluid next to it. */
int lb_set_geometry(lb_handle* h, int dom, const unsigned char* cls, const double* h_class,
                    int n_class);

/* Change the wall wetting gradients of domain dom between steps, keeping the
 * state (the quasi-static ramp of the wetting gradient in Sec. IV, by which
 * the paper moves a drop through a sequence of equilibrium angles).  Takes
 * effect from the next step; synchronises the stream.
 * Errors: LB_ERR_INVALID_ARG for non-finite gradients. */
int lb_set_wetting(lb_handle* h, int dom, double h_bottom, double h_top);

/* The obstacle map of domain dom (host [ny][nx]; all zero without one). */
int lb_get_geometry(lb_handle* h, int dom, unsigned char* cls);

/* Capillary filling set-up (Sec. VI) on a walled domain of nx x ny: the
 * columns x >= res_len are solid except the channel rows [y0, y0 + ch_w),
 * y0 = (ny - ch_w) / 2; the two solid rows bounding the channel are class 1
 * (gradient h_channel), every other solid node class 2 (h_block).  The
 * reservoir x < res_len connects to the channel outlet through the periodic
 * x boundary.  Initial phi: phase alpha (+1) in the reservoir columns
 * [res_len/2, res_len), beta (-1) elsewhere, flat tanh profiles
 * (l = sqrt(2 kappa / a)) centred half a node before columns res_len/2 and
 * res_len.  Then initialises as lb_init_phi.
 * Errors: LB_ERR_INVALID_ARG without walls, for res_len outside
 * [4, nx - 1], or a channel that leaves no solid row above or below it. */
int lb_init_channel(lb_handle* h, int dom, int res_len, int ch_w, double h_channel,
                    double h_block);

/* Meniscus in a horizontal channel with walls at the planes y_lo - 1/2 and
 * y_hi - 1/2 and phase alpha (phi > 0) behind it (smaller x), as in the
 * capillary set-up: the phi = 0 points (as lb_contact_angle) on links with
 * both ends in [x_lo, x_hi) x [y_lo, y_hi), farther than `exclude` from both
 * wall planes, fitted with a circle.  x_front: the circle's x on the channel
 * centre line, on the branch facing the points (l = x_front - (res_len -
 * 1/2) is the filled length of Eq. washburnlaw); theta_deg: the angle
 * through alpha at the walls (mean of both), the advancing angle theta^a of
 * Sec. VI while the front moves; R: the radius.  Any output may be NULL.
 * LB_ERR_NO_INTERFACE if fewer than 3 points remain. */
int lb_meniscus(lb_handle* h, int dom, int x_lo, int x_hi, int y_lo, int y_hi, double exclude,
                double* x_front, double* theta_deg, double* R);

/* Wetting gradient h that Eq. (theory) assigns to an equilibrium angle
 * theta (degrees, 0..180): sqrt(2 kappa/a) h = 2 sgn(theta - 90)
 * [cos(alpha/3)(1 - cos(alpha/3))]^(1/2), alpha = arccos(sin^2 theta).
 * Pure host arithmetic; returns NaN for arguments out of range. */
double lb_wetting_h(double theta_deg, double a, double kappa);

/* Absolute populations of domain dom as host arrays [9][ny][nx] (FP32 state
 * is widened to double).  Synchronises the stream. */
int lb_get_populations(lb_handle* h, int dom, double* f, double* g);

/* Rows [y0, y0 + nrows) only: host arrays [9][nrows][nx]. */
int lb_get_populations_rows(lb_handle* h, int dom, int y0, int nrows, double* f, double* g);

/* Overwrite domain dom's state with absolute populations (host arrays
 * [9][ny][nx]); FP32 storage rounds their deviations from the rest state.
 * The step count is left unchanged. */
int lb_set_populations(lb_handle* h, int dom, const double* f, const double* g);

/* Checkpoint: the exact device state of all domains plus the step count.
 * lb_state_bytes gives the size; save/load copy through a host buffer of at
 * least that size; a loaded state continues bit for bit. */
size_t lb_state_bytes(const lb_handle* h);
int lb_save_state(lb_handle* h, void* host_buf, size_t bytes);
int lb_load_state(lb_handle* h, const void* host_buf, size_t bytes);

/* Launch shape: threads per CTA along x (block_x, a multiple of 32 in
 * [32, 256], or [32, 288] with compact g storage) and rows each CTA marches
 * through (rows >= 1).  Results do not
 * depend on it.  On a batch it sets a one-class schedule with that shape
 * (lb_schedule).  Invalidates captured graphs. */
int lb_set_tile(lb_handle* h, int block_x, int rows);
int lb_get_tile(const lb_handle* h, int* block_x, int* rows);

/* Schedule of a batch (lb_create_batch; the configurations' many independent
 * domains, which the paper does not treat): how the (domain, strip, row
 * block) work of one time step is cut and spread over the GPU.
 *  n_class:     1..LB_MAX_SCHED_CLASSES domain-size classes.  Class k takes
 *               the domains with max_nx[k-1] < nx <= max_nx[k] (max_nx[-1] =
 *               0); the last class takes every wider domain (its max_nx is
 *               ignored).  Each class has its own launch per step.
 *  block_x[k], rows[k]: the launch shape of class k, as lb_set_tile (a
 *               strip of block_x columns, or with compact g storage two
 *               columns per compute thread less a 4-column halo, and `rows`
 *               rows per work item).
 *  ctas_per_sm[k]: 0 gives one CTA per work item (the hardware spreads
 *               them); n >= 1 a persistent grid of n CTAs per SM that take
 *               work items from a device counter.
 *  order:       0 work items by domain, then row block, then strip; 1
 *               largest item first (the small ragged items come last, which
 *               shortens the tail of each launch).
 *  chains:      with several classes, 1 lets each class advance through the
 *               steps of a captured graph as its own chain of launches
 *               (the classes hold disjoint domains, so they only meet at the
 *               graph's end); 0 launches the classes one after the other
 *               every step.
 *  persist:     1 runs all the steps of an lb_step call (of each captured
 *               graph of them) for a class in ONE launch of a persistent
 *               kernel (compact FP32 storage only): its CTAs take (step,
 *               work item) tickets in order from a device counter, and a
 *               work item's step waits, by a bounded spin on device flags,
 *               only for the items of its own domain that its halo reaches
 *               to finish the step before, not for the whole GPU.  Then
 *               ctas_per_sm[k] = 0 gives each class a share of the GPU in
 *               proportion to its rows (the classes, launched side by side,
 *               finish together); n >= 1 fixes n CTAs per SM.  A domain
 *               with obstacles (lb_set_geometry; any precision) likewise
 *               runs its steps as one cooperative launch of one CTA per
 *               tile, each tile waiting only for its neighbouring tiles,
 *               when all its tiles fit the GPU at once (else one launch per
 *               step).  A wait that gives up makes lb_step report
 *               LB_ERR_TIMEOUT.
 *  fill_pct:    persistent schedules: the shared-out CTAs of all classes
 *               fill this percentage of the GPU's registers, shared memory
 *               and thread slots (0 = 100; above 100 some CTAs wait for
 *               room and start when a class finishes).
 *  steps_per_launch: a single domain with obstacles (lb_set_geometry):
 *               2 runs two steps per launch (each CTA steps its tile and a
 *               four-node halo into shared memory, then its tile again; the
 *               halo is computed redundantly, no launch sits between the
 *               two steps); 0 or 1 one step per launch.  Ignored elsewhere
 *               and under persist.
 *  seal_edges[k]: compact storage: 1 makes class k's strips that cover
 *               their whole domain also zero the padding and (stale) ghost
 *               columns that share a 32-byte sector with their rows' first
 *               and last nodes, so that no sector is written in part (the
 *               memory reads a partly written sector before writing it
 *               back): a gain where memory bandwidth binds and rows are
 *               short, a few instructions more per row elsewhere.
 * Results do not depend on the schedule (bit for bit).  A single-domain
 * handle uses block_x[0] and rows[0] only.  Invalidates captured graphs.
 * Errors: LB_ERR_INVALID_ARG for a value out of range, max_nx not
 * increasing, persist on a batch without compact FP32 storage, fill_pct outside
 * [0, 400], steps_per_launch outside [0, 2], or a seal_edges value not 0
 * or 1. */
#define LB_MAX_SCHED_CLASSES 8
typedef struct lb_schedule {
    int n_class;
    int max_nx[LB_MAX_SCHED_CLASSES];
    int block_x[LB_MAX_SCHED_CLASSES];
    int rows[LB_MAX_SCHED_CLASSES];
    int ctas_per_sm[LB_MAX_SCHED_CLASSES];
    int order;
    int chains;
    int persist;
    int fill_pct;
    int steps_per_launch;
    int seal_edges[LB_MAX_SCHED_CLASSES];
} lb_schedule;
int lb_set_schedule(lb_handle* h, const lb_schedule* s);
int lb_get_schedule(const lb_handle* h, lb_schedule* s);

/* Autotuner: times each candidate for `reps` repetitions on the device
 * (without advancing the state) and keeps the fastest.  A single domain
 * tries launch shapes (block_x x rows); a single domain with obstacles, a
 * launch per step, two steps per launch and one persistent launch.  A batch tries schedules
 * (lb_schedule): one class, or ladders of size classes with their own strip
 * widths (sealed or not, per-step or persistent launches), rows per work
 * item, persistent or one-CTA-per-item grids, and the item order, each
 * timed as a captured graph of 16 steps, the fastest eight again over
 * 64-step graphs.  Outputs (class 0's shape and the best time per step in
 * ms) may be NULL; lb_get_schedule returns the whole choice. */
int lb_autotune(lb_handle* h, int reps, int* block_x, int* rows, double* best_ms);

/* Steps taken since the last initialisation (host-side count). */
long long lb_step_count(const lb_handle* h);

/* Synchronise the handle's stream.  LB_ERR_CUDA on a device error;
 * LB_ERR_TIMEOUT if a bounded device-side wait of an earlier step gave up
 * (its results are then invalid).  lb_moments reports the same. */
int lb_sync(lb_handle* h);

/* Number of kernel launches this handle has enqueued so far (graph replays
 * count every kernel node they run). */
long long lb_launch_count(const lb_handle* h);

const char* lb_error_string(int code);
const char* lb_last_error(void);

/* Self-check of the device-side wait bounds used by the step kernels (the
 * paper has no counterpart): one warp waits on a barrier that nothing ever
 * completes (the stage waits), another on a step flag that nothing ever
 * sets (the persistent batched kernel's wait for its neighbours); each wait
 * must give up after its wall-time bound (200 ms) and report it.  Returns
 * LB_ERR_TIMEOUT when both bounds work (the expected result), LB_OK if a
 * wait did not give up (a defect), LB_ERR_CUDA on a launch error.
 * Synchronises `stream`; leaves the context usable. */
int lb_check_wait_timeout(void* stream);

/* Measured FP64 throughput of the current device (the paper has no
 * counterpart: the roofline denominator of the FP64 build, which the FP64
 * pipe bounds).  A grid that fills the GPU runs independent dependency
 * chains of one operation -- kind 0 DFMA, 1 DADD, 2 DMUL -- and the
 * operations per second (a DFMA counts as one operation, two flops) over the
 * event-timed duration go to *ops_per_s.  Runs on `stream` (NULL = legacy
 * default) and synchronises it; allocates and frees a small buffer.
 * Errors: LB_ERR_INVALID_ARG for an unknown kind or a NULL output,
 * LB_ERR_CUDA on a CUDA failure. */
int lb_fp64_peak(int kind, void* stream, double* ops_per_s);

/* Diagnostics without any allocation (the paper has no counterpart: this is
 * a service for callers that may not allocate device memory at the time
 * they need the numbers -- an application that owns all device memory
 * through its own pool and forbids other allocations, or a long-running
 * service that must keep a fixed memory footprint).
 *  f, g:      device arrays [9][ny][nx] of absolute populations (the layout
 *             lb_get_populations returns), float for LB_FP32, double for
 *             LB_FP64; owned by the caller.
 *  stats_dev: device array of 6 doubles, owned by the caller, receiving
 *             sum rho, sum phi, sum rho u_x, sum rho u_y, max |u| and the
 *             number of nodes whose moments are not finite.
 * f, g and stats_dev must be device memory of one device; the work runs on
 * that device and is enqueued on `stream` (cudaStream_t of that device, NULL
 * = its legacy default stream); nothing is synchronised.  The calling
 * thread's current device is left as it was.  The scratch space is a fixed
 * device array of 1024 block partials (48 KiB) that the library carries on
 * every device it is loaded on until the process exits; its address is
 * looked up (a runtime query) on the first call made on a device.  All
 * calls share that array: calls that may
 * overlap on the GPU (unordered streams) race and can return wrong numbers.
 * At most LB_STATS_NOALLOC_MAX_VALUES population values per array
 * (9 * nx * ny); larger inputs, nx or ny < 1, NULL or non-device pointers,
 * arrays on different devices or an unknown precision give
 * LB_ERR_INVALID_ARG; a failed launch gives LB_ERR_CUDA (the launch status
 * itself: the runtime's last-error state is neither read nor cleared).  No
 * cudaMalloc, cudaFree or other allocating call is made. */
#define LB_STATS_NOALLOC_MAX_VALUES 2147483647LL
int lb_stats_noalloc(const void* f, const void* g, int nx, int ny, int precision,
                     double* stats_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBFE_H */
