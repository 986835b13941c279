// Kernels and their launchers: fused step (single domain and batched work
// list), initial state, moments / diagnostics and interface points.
#include <cuda_runtime.h>

#include <cstdint>

#include "lb_internal.h"
#include "lb_node.cuh"
#include "lb_step_kernels.cuh"

namespace lbfe {

// ------------------------------------------------------------------ step
// The step kernels live in lb_step_kernels.cuh, instantiated per precision in
// lb_step_f32.cu and lb_step_f64.cu (compiled in parallel).

size_t step_smem_bytes(int precision, int bx)
{
    if (bx < 32 || bx > 256 || bx % 32) return 0;
    return precision == 0 ? StageLayout<float>(bx / 32, kStages<float>).total()
                          : StageLayout<double>(bx / 32, kStages<double>).total();
}

int prepare_step_kernels()
{
    int e = prepare_step_f32();
    if (e == 0) e = prepare_step_f64();
    if (e == 0) e = prepare_persist();
    return e;
}

int launch_step(int precision, int coll, const DomDesc& d, const DomDesc* d_descs,
                const WorkItem* d_items, int n_items, int n_dom, int parity, int block_x, int rows,
                int band_mul, int grid_persistent, int* sched, bool one_body, void* stream)
{
    const bool ok = d.compact ? (block_x >= 32 && block_x <= 288 && block_x % 32 == 0)
                              : step_smem_bytes(precision, block_x) != 0;
    if (!ok) return int(cudaErrorInvalidValue);
    return precision == 0
               ? launch_step_f32(coll, d, d_descs, d_items, n_items, n_dom, parity, block_x, rows,
                                 band_mul, grid_persistent, sched, one_body, stream)
               : launch_step_f64(coll, d, d_descs, d_items, n_items, n_dom, parity, block_x, rows,
                                 band_mul, grid_persistent, sched, one_body, stream);
}

static int step_occupancy(int precision, int coll, int compact, int block_x, int single)
{
    if (compact ? (block_x < 32 || block_x > 288 || block_x % 32) : step_smem_bytes(precision, block_x) == 0)
        return 0;
    return precision == 0 ? batch_occupancy_f32(coll, compact, block_x, single)
                          : batch_occupancy_f64(coll, block_x, single);
}

int step_batch_occupancy(int precision, int coll, int compact, int block_x)
{
    return step_occupancy(precision, coll, compact, block_x, 0);
}

int step_single_occupancy(int precision, int coll, int compact, int block_x)
{
    return step_occupancy(precision, coll, compact, block_x, 1);
}

// Periodic ghost columns of every row of the 18 planes of one buffer, from
// the logical columns they mirror (used after host writes).
template <typename Real>
__global__ void fill_ghosts_kernel(DomDesc D, int parity)
{
    Real* f = static_cast<Real*>(parity ? D.f[1] : D.f[0]);
    Real* g = static_cast<Real*>(parity ? D.g[1] : D.g[0]);
    const long long rows = 9LL * D.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < 2 * rows * 4;
         k += (long long)gridDim.x * blockDim.x) {
        const int which = int(k & 3);        // ghost column: -2, -1, nx, nx+1
        const long long rr = (k >> 2) % rows;  // plane * ny + row
        Real* base = ((k >> 2) < rows ? f : g) + rr * D.pitch + kXOff;
        const int dst = which < 2 ? which - 2 : D.nx + (which - 2);
        const int src = which < 2 ? D.nx + which - 2 : which - 2;
        base[dst] = base[src];
    }
}

int launch_fill_ghosts(int precision, const DomDesc& d, int parity, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == 0)
        fill_ghosts_kernel<float><<<64, 256, 0, s>>>(d, parity);
    else
        fill_ghosts_kernel<double><<<64, 256, 0, s>>>(d, parity);
    return static_cast<int>(cudaGetLastError());
}

// ------------------------------------------------------------ init phi0
// phi0 is a double field with the domain's pitch (it lives in the idle
// ping-pong buffer during initialisation).
__global__ void init_phi_drop_kernel(int nx, int ny, int pitch, double* phi0, double R, double cx,
                                     double cy, double ell)
{
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = int(k / nx), x = int(k - (long long)y * nx);
        const double ddx = x - cx, ddy = y - cy;
        phi0[(long long)y * pitch + x] = tanh((R - sqrt(ddx * ddx + ddy * ddy)) / ell);
    }
}

// SplitMix64 used as a counter-based generator (Steele, Lea & Flood 2014):
// draw k of the stream seeded with s is mix(s + (k + 1) * golden gamma).
__device__ __forceinline__ unsigned long long splitmix64_draw(unsigned long long seed,
                                                              unsigned long long k)
{
    unsigned long long z = seed + (k + 1ULL) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void init_phi_random_kernel(int nx, int ny, int pitch, double* phi0, double amp,
                                       unsigned long long seed)
{
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = int(k / nx), x = int(k - (long long)y * nx);
        const double u = double(splitmix64_draw(seed, (unsigned long long)k) >> 11) * 0x1.0p-53;
        phi0[(long long)y * pitch + x] = amp * (2.0 * u - 1.0);
    }
}

static int grid_for(long long n, int block)
{
    long long g = (n + block - 1) / block;
    if (g > 152LL * 16) g = 152LL * 16;
    if (g < 1) g = 1;
    return int(g);
}

int launch_init_phi_drop(int, const DomDesc& d, double* phi0, double R, double cx, double cy,
                         void* stream)
{
    const double ell = sqrt(2.0 * d.kappa / d.a);
    const long long n = (long long)d.nx * d.ny;
    init_phi_drop_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d.nx, d.ny, d.pitch, phi0, R, cx, cy, ell);
    return static_cast<int>(cudaGetLastError());
}

// Rows of a caller's phi0 (nx per row, contiguous; page-locked host memory
// seen through its device address) into the pitched scratch field.
__global__ void copy_rows_kernel(const double* __restrict__ src, int nx, int ny,
                                 double* __restrict__ dst, int pitch)
{
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = int(k / nx), x = int(k - (long long)y * nx);
        dst[(long long)y * pitch + x] = src[k];
    }
}

int launch_copy_rows(const DomDesc& d, const double* src, double* phi0, void* stream)
{
    const long long n = (long long)d.nx * d.ny;
    copy_rows_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        src, d.nx, d.ny, phi0, d.pitch);
    return static_cast<int>(cudaGetLastError());
}

int launch_init_phi_random(int, const DomDesc& d, double* phi0, double amp,
                           unsigned long long seed, void* stream)
{
    const long long n = (long long)d.nx * d.ny;
    init_phi_random_kernel<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d.nx, d.ny, d.pitch, phi0, amp, seed);
    return static_cast<int>(cudaGetLastError());
}

// f = f^eq, g = g^eq of (rho = 1, u = 0, phi0) with the stencils of Eq.
// (best) and the wetting ghost rows; computed in FP64, stored as Real.
template <typename Real>
__global__ void init_eq_kernel(DomDesc D, const double* __restrict__ phi0, int parity)
{
    Real* fd = static_cast<Real*>((parity ? D.f[1] : D.f[0]));
    Real* gd = static_cast<Real*>((parity ? D.g[1] : D.g[0]));
    const int nx = D.nx, ny = D.ny, pitch = D.pitch;
    const long long P = D.plane;
    NodeParams<double> prm;
    prm.a = D.a;
    prm.kappa = D.kappa;
    prm.gamma = D.gamma;
    prm.omega_phi = D.omega_phi;
    prm.tau_c0 = D.tau_c0;
    prm.tau_c1 = D.tau_c1;
    prm.h_bot = D.h_bot;
    prm.h_top = D.h_top;
    prm.lut_lo = prm.lut_step = prm.lut_inv = prm.lut_kmax = 0.0;  // no collision here
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = int(k / nx), x = int(k - (long long)y * nx);
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x + 1 == nx ? 0 : x + 1;
        // phi in rows y-1, y, y+1 at columns xm, x, xp
        double v[3][3];
        for (int r = 0; r < 3; ++r) {
            const int yy = y + r - 1;
            const int cols[3] = {xm, x, xp};
            for (int c = 0; c < 3; ++c) {
                double val;
                if (D.walls && yy < 0)
                    val = phi0[(long long)(D.wet_k - 1) * pitch + cols[c]] - D.wet_k * D.h_bot;
                else if (D.walls && yy >= ny)
                    val = phi0[(long long)(ny - D.wet_k) * pitch + cols[c]] - D.wet_k * D.h_top;
                else {
                    const int yw = yy < 0 ? ny - 1 : (yy >= ny ? 0 : yy);
                    val = phi0[(long long)yw * pitch + cols[c]];
                }
                v[r][c] = val;
            }
        }
        const double phi = v[1][1];
        double fe[9], ge[9], G;
        if constexpr (sizeof(Real) == 4) {
            // FP32 storage: the stencils and equilibria in FP32 (the result is
            // rounded to FP32 anyway; this GPU's FP64 pipe is 1/64 of the FP32
            // rate), phi and g_0 from the FP64 input
            const NodeParams<float> pf = node_params<float>(D);
            float vf[3][3];
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) vf[r][c] = float(v[r][c]);
            float dxf, dyf, lapf, fef[9], gef[9], m7f, m8f;
            stencils<float>(vf[1][1], vf[1][2], vf[1][0], vf[2][1], vf[0][1], vf[2][2], vf[2][0],
                            vf[0][2], vf[0][0], dxf, dyf, lapf);
            equilibria<float>(pf, 0.f, vf[1][1], 0.f, 0.f, 0.f, 0.f, dxf, dyf, lapf, fef, gef, m7f,
                              m8f);
            fef[0] = -((((fef[1] + fef[2]) + (fef[3] + fef[4])) + ((fef[5] + fef[6]) + (fef[7] + fef[8]))));
            for (int i = 0; i < 9; ++i) {
                fe[i] = fef[i];
                ge[i] = gef[i];
            }
            ge[0] = phi - double(g_tail_sum<float>(gef));
            G = gamma_mu<float>(pf, vf[1][1], lapf);
        } else {
            double dx, dy, lap, m7eq, m8eq;
            stencils<double>(v[1][1], v[1][2], v[1][0], v[2][1], v[0][1], v[2][2], v[2][0], v[0][2],
                             v[0][0], dx, dy, lap);
            equilibria<double>(prm, 0.0, phi, 0.0, 0.0, 0.0, 0.0, dx, dy, lap, fe, ge, m7eq, m8eq);
            fe[0] = -((((fe[1] + fe[2]) + (fe[3] + fe[4])) + ((fe[5] + fe[6]) + (fe[7] + fe[8]))));
            ge[0] = phi - ((((ge[1] + ge[2]) + (ge[3] + ge[4])) + ((ge[5] + ge[6]) + (ge[7] + ge[8]))));
            G = gamma_mu<double>(prm, phi, lap);
        }
        const long long o = (long long)y * pitch + x + kXOff;
        const long long og1 = x < 2 ? o + nx : -1, og2 = x >= nx - 2 ? o - nx : -1;
        // compact g storage: (phi word, Gamma mu, u_eq = 0) in planes 0..3
        const double cg[4] = {0.0, G, 0.0, 0.0};
        for (int i = 0; i < 9; ++i) {
            const Real fv = Real(fe[i]);
            Real gv;
            if (D.compact)
                gv = i == 0 ? G0<Real>::encode(phi) : Real(i < 4 ? cg[i] : 0.0);
            else
                gv = i == 0 ? G0<Real>::encode(ge[0]) : Real(ge[i]);
            fd[i * P + o] = fv;
            gd[i * P + o] = gv;
            if (og1 >= 0) {
                fd[i * P + og1] = fv;
                gd[i * P + og1] = gv;
            }
            if (og2 >= 0) {
                fd[i * P + og2] = fv;
                gd[i * P + og2] = gv;
            }
        }
    }
}

int launch_init_eq(int precision, const DomDesc& d, const double* phi0, int parity, void* stream)
{
    const long long n = (long long)d.nx * d.ny;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == 0)
        init_eq_kernel<float><<<grid_for(n, 256), 256, 0, s>>>(d, phi0, parity);
    else
        init_eq_kernel<double><<<grid_for(n, 256), 256, 0, s>>>(d, phi0, parity);
    return static_cast<int>(cudaGetLastError());
}

// ------------------------------------------------------------- moments
// Moments of the stored populations (Eq. moments) on rows
// [row0, row0 + nrows): optional FP64 field outputs (leading dimension ld,
// row-relative), and per-block partial sums for the diagnostics.
// Reductions: fixed grid, per-thread serial accumulation, warp shuffles,
// one partial per block, then a single-block pass in fixed order, so the
// result is deterministic.
constexpr int kMomBlock = 256;
constexpr int kMaxMomBlocks = 4096;  // ~27 blocks of 256 per SM: enough loads in flight

int max_partials_needed(int, int) { return kMaxMomBlocks; }

__device__ __forceinline__ void warp_reduce(double (&v)[kStatsFields])
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int k = 0; k < kStatsFields; ++k) {
            const double o = __shfl_xor_sync(0xffffffffu, v[k], off);
            v[k] = (k == 4) ? fmax(v[k], o) : v[k] + o;
        }
    }
}

template <typename Real>
__global__ void __launch_bounds__(kMomBlock) moments_kernel(DomDesc D, int parity, int row0,
                                                            int nrows, double* rho, double* phi,
                                                            double* ux, double* uy, long long ld,
                                                            double* partials)
{
    const Real* fs = static_cast<const Real*>((parity ? D.f[1] : D.f[0]));
    const Real* gs = static_cast<const Real*>((parity ? D.g[1] : D.g[0]));
    const long long P = D.plane;
    const int nx = D.nx, pitch = D.pitch;
    const long long n = (long long)nx * nrows;
    double acc[kStatsFields] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if constexpr (sizeof(Real) == 4) {
        // FP32 storage: per-node arithmetic in FP32 and per-thread sums of the
        // small quantities (rho - 1, rho u, the g tail) in FP32, of the phi
        // words as exact 64-bit integers; widened once per thread (this GPU's
        // FP64 pipe runs at 1/64 of the FP32 rate)
        float s_drho = 0.f, s_jx = 0.f, s_jy = 0.f, s_tail = 0.f, s_um = 0.f;
        long long s_word = 0, s_n = 0;
        int s_bad = 0;
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
             k += (long long)gridDim.x * blockDim.x) {
            const int yr = int(k / nx), x = int(k - (long long)yr * nx);
            const long long q = (long long)yr * ld + x;
            if (D.cls && D.cls[(long long)(row0 + yr) * nx + x] != 0) {
                // solid node: no fluid, no contribution to the diagnostics
                if (rho) rho[q] = 0.0;
                if (phi) phi[q] = 0.0;
                if (ux) ux[q] = 0.0;
                if (uy) uy[q] = 0.0;
                continue;
            }
            const long long o = (long long)(row0 + yr) * pitch + x + kXOff;
            float f[9];
            for (int i = 0; i < 9; ++i) f[i] = float(fs[i * P + o]);
            const float drho = (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]))) + f[8];
            const float jxf = (f[1] - f[2]) + (f[5] - f[6]) + (f[8] - f[7]);
            const float jyf = (f[3] - f[4]) + (f[5] - f[6]) + (f[7] - f[8]);
            float tail = 0.f;
            if (!D.compact) {
                float g[9];
                for (int i = 1; i < 9; ++i) g[i] = float(gs[i * P + o]);
                tail = g_tail_sum<float>(g);
            }
            const float word_raw = float(gs[o]);
            const float rf = 1.f + drho;
            const float vxf = jxf / rf, vyf = jyf / rf;
            const float umf = sqrtf(vxf * vxf + vyf * vyf);
            if (rho) rho[q] = 1.0 + double(drho);
            if (phi) phi[q] = G0<float>::decode(word_raw) + double(tail);
            if (ux) ux[q] = double(vxf);
            if (uy) uy[q] = double(vyf);
            const bool finite = isfinite(drho) && isfinite(tail) && isfinite(umf);
            s_drho += drho;
            s_jx += jxf;
            s_jy += jyf;
            s_tail += tail;
            s_word += __float_as_int(word_raw);
            ++s_n;
            s_um = finite ? fmaxf(s_um, umf) : s_um;
            s_bad += finite ? 0 : 1;
        }
        acc[0] = double(s_n) + double(s_drho);
        acc[1] = double(s_word) / G0<float>::kScale + double(s_tail);
        acc[2] = double(s_jx);
        acc[3] = double(s_jy);
        acc[4] = double(s_um);
        acc[5] = double(s_bad);
    } else {
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
             k += (long long)gridDim.x * blockDim.x) {
            const int yr = int(k / nx), x = int(k - (long long)yr * nx);
            const long long q = (long long)yr * ld + x;
            if (D.cls && D.cls[(long long)(row0 + yr) * nx + x] != 0) {
                if (rho) rho[q] = 0.0;
                if (phi) phi[q] = 0.0;
                if (ux) ux[q] = 0.0;
                if (uy) uy[q] = 0.0;
                continue;
            }
            const long long o = (long long)(row0 + yr) * pitch + x + kXOff;
            double f[9], g[9];
            for (int i = 0; i < 9; ++i) f[i] = double(fs[i * P + o]);
            g[0] = G0<Real>::decode(gs[o]);
            for (int i = 1; i < 9; ++i) g[i] = D.compact ? 0.0 : double(gs[i * P + o]);
            const double drho = (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]))) + f[8];
            const double jx = (f[1] - f[2]) + (f[5] - f[6]) + (f[8] - f[7]);
            const double jy = (f[3] - f[4]) + (f[5] - f[6]) + (f[7] - f[8]);
            const double ph = phi_sum<double>(g);
            const double r = 1.0 + drho;
            const double vx = jx / r, vy = jy / r;
            if (rho) rho[q] = r;
            if (phi) phi[q] = ph;
            if (ux) ux[q] = vx;
            if (uy) uy[q] = vy;
            const double um = sqrt(vx * vx + vy * vy);
            const bool finite = isfinite(r) && isfinite(ph) && isfinite(um);
            acc[0] += r;
            acc[1] += ph;
            acc[2] += jx;
            acc[3] += jy;
            acc[4] = finite ? fmax(acc[4], um) : acc[4];
            acc[5] += finite ? 0.0 : 1.0;
        }
    }
    if (partials == nullptr) return;
    warp_reduce(acc);
    __shared__ double red[kMomBlock / 32][kStatsFields];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < kStatsFields; ++k) red[wid][k] = acc[k];
    __syncthreads();
    if (wid == 0) {
        double v[kStatsFields];
        for (int k = 0; k < kStatsFields; ++k)
            v[k] = lane < (kMomBlock / 32) ? red[lane][k] : (k == 4 ? 0.0 : 0.0);
        warp_reduce(v);
        if (lane == 0)
            for (int k = 0; k < kStatsFields; ++k) partials[blockIdx.x * kStatsFields + k] = v[k];
    }
}

__global__ void finalize_stats_kernel(const double* __restrict__ partials, int nblocks,
                                      StatsOut* out)
{
    double acc[kStatsFields] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < kStatsFields; ++k) {
            const double v = partials[b * kStatsFields + k];
            acc[k] = (k == 4) ? fmax(acc[k], v) : acc[k] + v;
        }
    warp_reduce(acc);
    __shared__ double red[32][kStatsFields];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < kStatsFields; ++k) red[wid][k] = acc[k];
    __syncthreads();
    if (wid == 0) {
        double v[kStatsFields];
        const int nw = blockDim.x >> 5;
        for (int k = 0; k < kStatsFields; ++k) v[k] = lane < nw ? red[lane][k] : 0.0;
        warp_reduce(v);
        if (lane == 0) {
            out->mass = v[0];
            out->order = v[1];
            out->mom_x = v[2];
            out->mom_y = v[3];
            out->max_u = v[4];
            out->nonfinite = v[5];
        }
    }
}

int launch_moments(int precision, const DomDesc& d, int parity, int row0, int nrows, double* rho,
                   double* phi, double* ux, double* uy, long long ld, double* partials,
                   int max_partials, StatsOut* out, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long n = (long long)d.nx * nrows;
    long long g = (n + kMomBlock - 1) / kMomBlock;
    if (g > kMaxMomBlocks) g = kMaxMomBlocks;
    if (out && g > max_partials) g = max_partials;
    if (g < 1) g = 1;
    const int grid = int(g);
    double* part = out ? partials : nullptr;
    if (precision == 0)
        moments_kernel<float><<<grid, kMomBlock, 0, s>>>(d, parity, row0, nrows, rho, phi, ux, uy,
                                                         ld, part);
    else
        moments_kernel<double><<<grid, kMomBlock, 0, s>>>(d, parity, row0, nrows, rho, phi, ux,
                                                          uy, ld, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || out == nullptr) return static_cast<int>(e);
    finalize_stats_kernel<<<1, 256, 0, s>>>(partials, grid, out);
    return static_cast<int>(cudaGetLastError());
}

// ----------------------------------------------------- interface points
// phi = 0 crossings on horizontal (periodic) and vertical links whose ends
// have phi > 0 and phi < 0, by linear interpolation (Sec. IV); links that
// touch a solid node are skipped.  Points are appended in arbitrary order;
// the host sorts them.
template <typename Real>
__device__ __forceinline__ double phi_at_node(const Real* g, long long P, long long o,
                                              bool compact)
{
    if (compact) return G0<Real>::decode(g[o]);  // the phi word itself
    double v[9];
    v[0] = G0<Real>::decode(g[o]);
    for (int i = 1; i < 9; ++i) v[i] = double(g[i * P + o]);
    return phi_sum<double>(v);
}

template <typename Real>
__global__ void crossings_kernel(DomDesc D, int parity, double* pts, int* count, int cap)
{
    const Real* gs = static_cast<const Real*>((parity ? D.g[1] : D.g[0]));
    const long long P = D.plane;
    const int nx = D.nx, ny = D.ny, pitch = D.pitch;
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = int(k / nx), x = int(k - (long long)y * nx);
        const unsigned char* cls = D.cls;
        if (cls && cls[k] != 0) continue;  // links touching a solid node carry no interface
        const bool cmp = D.compact != 0;
        const double a = phi_at_node(gs, P, (long long)y * pitch + x + kXOff, cmp);
        const int xp = x + 1 == nx ? 0 : x + 1;
        const double b = phi_at_node(gs, P, (long long)y * pitch + xp + kXOff, cmp);
        const bool bfluid = !cls || cls[(long long)y * nx + xp] == 0;
        if (bfluid && ((a > 0.0 && b < 0.0) || (a < 0.0 && b > 0.0))) {
            const int idx = atomicAdd(count, 1);
            if (idx < cap) {
                pts[2 * idx] = x + a / (a - b);
                pts[2 * idx + 1] = double(y);
            }
        }
        if (y + 1 < ny && (!cls || cls[(long long)(y + 1) * nx + x] == 0)) {
            const double c = phi_at_node(gs, P, (long long)(y + 1) * pitch + x + kXOff, cmp);
            if ((a > 0.0 && c < 0.0) || (a < 0.0 && c > 0.0)) {
                const int idx = atomicAdd(count, 1);
                if (idx < cap) {
                    pts[2 * idx] = double(x);
                    pts[2 * idx + 1] = y + a / (a - c);
                }
            }
        }
    }
}

int launch_crossings(int precision, const DomDesc& d, int parity, double* pts, int* count, int cap,
                     void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
    if (e != cudaSuccess) return static_cast<int>(e);
    const long long n = (long long)d.nx * d.ny;
    if (precision == 0)
        crossings_kernel<float><<<grid_for(n, 256), 256, 0, s>>>(d, parity, pts, count, cap);
    else
        crossings_kernel<double><<<grid_for(n, 256), 256, 0, s>>>(d, parity, pts, count, cap);
    return static_cast<int>(cudaGetLastError());
}

// ------------------------------------------------ bounded-wait self-check
// Warp 0 waits on an mbarrier that nothing ever completes (the stage waits
// of the step kernels), warp 1 on a step flag that nothing ever sets (the
// persistent batched kernel's wait for neighbouring work items).  Each wait
// must give up after its wall-time bound and record the failure in its own
// word.
static __device__ unsigned g_selfcheck_err[2];
static __device__ int g_selfcheck_flag;

__global__ void wait_selfcheck_kernel()
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x < 32)
        mbar_wait(&bar, 0, &g_selfcheck_err[0]);
    else
        flag_wait(&g_selfcheck_flag, 1, &g_selfcheck_err[1]);
}

int run_wait_selfcheck(void* stream, unsigned* word)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned zero[2] = {0, 0};
    const int zflag = 0;
    cudaError_t e = cudaMemcpyToSymbolAsync(g_selfcheck_err, zero, sizeof(zero), 0,
                                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbolAsync(g_selfcheck_flag, &zflag, sizeof(zflag), 0,
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return int(e);
    wait_selfcheck_kernel<<<1, 64, 0, s>>>();
    if ((e = cudaGetLastError()) != cudaSuccess) return int(e);
    unsigned got[2] = {0, 0};
    e = cudaMemcpyFromSymbolAsync(got, g_selfcheck_err, sizeof(got), 0, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return int(e);
    e = cudaStreamSynchronize(s);
    // bit 0: the barrier wait gave up, bit 1: the flag wait gave up
    *word = (got[0] ? 1u : 0u) | (got[1] ? 2u : 0u);
    return int(e);
}

}  // namespace lbfe
