// Time step of a domain with solid obstacles (capillary filling, Sec. VI).
//
// The paper states bounce-back and the wetting boundary condition for flat
// walls only; on an obstacle map they are read node by node:
//   - a population whose pull source r - e_i is solid is the node's own
//     reversed post-collision population (mid-link bounce-back, as at walls);
//   - Step 2 (zero equilibrium velocity) applies to fluid nodes with a solid
//     node among their eight neighbours;
//   - a solid node s next to fluid carries the wetting ghost value: the
//     flat-wall mirror phi(s + 2d) - 2 h(s) (or, with the one-sided rule,
//     phi(s + d) - h(s)), averaged over the axis directions d whose
//     neighbour s + d is fluid, or over the diagonal directions if s
//     touches fluid only through a corner.  The host rejects
//     maps where a mirror node s + 2d is solid (features thinner than two
//     nodes).  On an obstacle-free lattice this is the ghost-row rule of the
//     plain step, so both paths agree there.
// With walls, the rows y = -1 and y = ny are solid with h_bot / h_top.
//
// Node bounce-back (the paper's Fig. 4b, the wall on the boundary nodes),
// class kNodeWall in row 0 or ny - 1 of a walled domain, read as the
// full-way scheme: a wall node streams like a fluid node (its pulls from
// beyond the domain bounce back) and reverses every population instead of
// colliding; its fluid neighbours see phi(x, 0) = phi(x, 1) - h_bot (phi(x,
// ny-1) = phi(x, ny-2) - h_top) and are Step-2 nodes.
//
// A step is one launch.  A CTA owns a tile of kGTX x kGTY nodes (one per
// thread) and, in shared memory:
//   1. the class map of the tile and a kGC-node halo;
//   2. phi of the tile and a kGH-node halo, each fluid node's sum of its
//      pulled g (Eq. moments): a ghost value at a solid neighbour reads phi
//      up to three nodes from the fluid node it serves (the solid node, then
//      twice the direction towards fluid), and the pulls of the halo reach
//      one node further;
// then each fluid node of the tile pulls f and g, takes the phi stencil
// from shared memory (ghost values at solid neighbours), collides (the node
// arithmetic of the plain step) and stores.  Halo nodes are formed by
// several CTAs with the same arithmetic, so every tile sees the same phi.
// Solid nodes are never written by a step; they hold the rest state
// (f = t, g = 0), so they carry no fluid.
//
// The obstacle path serves small and medium geometries (the capillary set-up
// is ~10^5 nodes) whose state stays in L2: a step is bound by launch and L2
// latency rather than by HBM bandwidth, so it uses plain loads instead of
// the staged pipeline of the plain step, and one launch with one shared
// phi field instead of a phi pass through memory.
#include <cuda_runtime.h>

#include "lb_async.cuh"
#include "lb_internal.h"
#include "lb_geo_persist.h"
#include "lb_node.cuh"

namespace lbfe {

namespace {

constexpr int kGeoBlock = 128;

template <typename Real>
__device__ __forceinline__ NodeParams<Real> geo_params(const DomDesc& D);
template <>
__device__ __forceinline__ NodeParams<float> geo_params<float>(const DomDesc& D)
{
    return NodeParams<float>{D.fa,      D.fkappa,  D.fgamma,   D.fomega_phi,
                             D.ftau_c0, D.ftau_c1, D.fh_bot,   D.fh_top,
                             D.flut_lo, D.flut_step, D.flut_inv, D.flut_kmax};
}
template <>
__device__ __forceinline__ NodeParams<double> geo_params<double>(const DomDesc& D)
{
    return NodeParams<double>{D.a,      D.kappa,  D.gamma,   D.omega_phi,
                              D.tau_c0, D.tau_c1, D.h_bot,   D.h_top,
                              D.lut_lo, D.lut_step, D.lut_inv, D.lut_kmax};
}

template <typename Real>
__device__ __forceinline__ Real class_h(const DomDesc& D, int k);
template <>
__device__ __forceinline__ float class_h<float>(const DomDesc& D, int k)
{
    return D.fhcls[k];
}
template <>
__device__ __forceinline__ double class_h<double>(const DomDesc& D, int k)
{
    return D.hcls[k];
}

// periodic index for offsets of a few nodes (|v| < 2n)
__device__ __forceinline__ int wrap_near(int v, int n)
{
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

// velocity components in the paper's order
__device__ __forceinline__ int gex(int i)
{
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 2 || i == 6 || i == 7) ? -1 : 0);
}
__device__ __forceinline__ int gey(int i)
{
    return (i == 3 || i == 5 || i == 7) ? 1 : ((i == 4 || i == 6 || i == 8) ? -1 : 0);
}
__device__ __forceinline__ int gopp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

struct GeoView {
    const unsigned char* cls;
    int nx, ny, walls;

    // wetting class of (x, y); 0 = fluid, -1 / -2 = the bottom / top wall row
    __device__ __forceinline__ int cls_at(int x, int y) const
    {
        if (walls && y < 0) return -1;
        if (walls && y >= ny) return -2;
        return cls[(long long)wrap_near(y, ny) * nx + wrap_near(x, nx)];
    }
    __device__ __forceinline__ bool solid(int x, int y) const { return cls_at(x, y) != 0; }
};

// Tile of the fused obstacle step and its halos.
constexpr int kGTX = 32, kGTY = 8;  // nodes of one CTA (one per thread)
constexpr int kGH = 3;              // phi halo
constexpr int kGC = kGH + 1;        // class-map halo
constexpr int kGCX = kGTX + 2 * kGC, kGCY = kGTY + 2 * kGC;
constexpr int kGPX = kGTX + 2 * kGH, kGPY = kGTY + 2 * kGH;

// periodic index for any offset (halos may exceed a small lattice)
__device__ __forceinline__ int wrap_any(int v, int n)
{
    const int r = v % n;
    return r < 0 ? r + n : r;
}

// Per-CTA tables of a tile: the wrapped halo coordinates and the class map
// with its halo.  They depend only on the geometry, so the persistent form
// builds them once per launch.
struct GeoTables {
    int colx[kGCX];  // wrapped column (+ kXOff) of each halo column
    int rowo[kGCY];  // offset of each halo row (wrapped row x pitch)
    int rowc[kGCY];  // the same row in the class map (wrapped row x nx)
    signed char cl[kGCY][kGCX];  // 0 fluid, k > 0 solid class k, -1 / -2 wall rows
};

__device__ __forceinline__ void geo_tile_setup(const DomDesc& D, int x0, int y0, GeoTables& t)
{
    const int nx = D.nx, ny = D.ny;
    // 0. periodic wrap of the halo coordinates
    for (int k = threadIdx.x; k < kGCX + kGCY; k += blockDim.x) {
        if (k < kGCX)
            t.colx[k] = wrap_any(x0 - kGC + k, nx) + kXOff;
        else {
            const int wy = wrap_any(y0 - kGC + (k - kGCX), ny);
            t.rowo[k - kGCX] = wy * D.pitch;
            t.rowc[k - kGCX] = wy * nx;
        }
    }
    __syncthreads();
    // 1. class map (0 fluid, k > 0 solid class k, -1 / -2 bottom / top wall row)
    for (int k = threadIdx.x; k < kGCX * kGCY; k += blockDim.x) {
        const int cy = k / kGCX, cx = k - cy * kGCX;
        const int y = y0 - kGC + cy;
        int c;
        if (D.walls && y < 0)
            c = -1;
        else if (D.walls && y >= ny)
            c = -2;
        else
            c = D.cls[t.rowc[cy] + (t.colx[cx] - kXOff)];
        t.cl[cy][cx] = static_cast<signed char>(c);
    }
    __syncthreads();
}

// Load of a stored population: through L1, or (L2ONLY, the persistent form,
// whose neighbours rewrite the state within the launch) from L2.
template <bool L2ONLY, typename Real>
__device__ __forceinline__ Real geo_ld(const Real* p)
{
    if constexpr (L2ONLY)
        return __ldcg(p);
    else
        return *p;
}

// The step of one fluid or wall node (x, y) of class cme from its pulled
// populations f, g: cls_l(x, y) reads the class map and phi_l(x, y) phi of
// the same state around the node (lattice coordinates; ghost values at solid
// neighbours reach three nodes away); fo, go receive the new populations.
template <typename Real, bool MRT, class ClsF, class PhiF>
__device__ __forceinline__ void geo_node_update(const DomDesc& D, int x, int y, int cme,
                                                const Real (&f)[9], const Real (&g)[9], ClsF cls_l,
                                                PhiF phi_l, Real (&fo)[9], Real (&go)[9])
{
    const int ny = D.ny;
    if (cme == kNodeWall) {
        // node bounce-back: every population reversed, no collision
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            fo[i] = f[gopp(i)];
            go[i] = g[gopp(i)];
        }
        return;
    }
    const Real c = phi_sum<Real>(g);
    // wetting ghost value of solid node (sx, sy): the mean over the axis (or,
    // through a corner only, the diagonal) directions d towards fluid of
    // phi(s + k d) - k h, k = D.wet_k
    auto ghost = [&](int sx, int sy) -> Real {
        const int k = cls_l(sx, sy);
        const Real h = k == -1 ? (sizeof(Real) == 4 ? Real(D.fh_bot) : Real(D.h_bot))
                     : k == -2 ? (sizeof(Real) == 4 ? Real(D.fh_top) : Real(D.h_top))
                               : class_h<Real>(D, k);
        Real sum = Real(0);
        int n = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int dx = j == 0 ? 1 : (j == 1 ? -1 : 0);
            const int dy = j == 2 ? 1 : (j == 3 ? -1 : 0);
            if (cls_l(sx + dx, sy + dy) == 0) {
                sum += phi_l(sx + D.wet_k * dx, sy + D.wet_k * dy);
                ++n;
            }
        }
        if (n == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int dx = (j == 0 || j == 3) ? 1 : -1;
                const int dy = (j == 0 || j == 2) ? 1 : -1;
                if (cls_l(sx + dx, sy + dy) == 0) {
                    sum += phi_l(sx + D.wet_k * dx, sy + D.wet_k * dy);
                    ++n;
                }
            }
        }
        const Real mean = n == 1 ? sum : (n == 2 ? sum * Real(0.5) : (n == 3 ? div_const<3>(sum) : sum * Real(0.25)));
        return mean - Real(D.wet_k) * h;
    };
    // phi at the eight neighbours; ghost values at solid ones
    Real nb[9];
    bool next_to_solid = false;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int qx = x + gex(i), qy = y + gey(i);
        const int cq = cls_l(qx, qy);
        if (cq == kNodeWall) {
            // one-sided wetting value from the first fluid row
            next_to_solid = true;
            nb[i] = qy == 0 ? phi_l(qx, 1) - (sizeof(Real) == 4 ? Real(D.fh_bot) : Real(D.h_bot))
                            : phi_l(qx, ny - 2) - (sizeof(Real) == 4 ? Real(D.fh_top) : Real(D.h_top));
        } else if (cq != 0) {
            next_to_solid = true;
            nb[i] = ghost(qx, qy);
        } else {
            nb[i] = phi_l(qx, qy);
        }
    }
    Real dx, dy, lap;
    // order: centre, E, W, N, S, NE, NW, SE, SW
    stencils<Real>(c, nb[1], nb[2], nb[3], nb[4], nb[5], nb[7], nb[8], nb[6], dx, dy, lap);
    const NodeParams<Real> prm = geo_params<Real>(D);
    collide<Real, MRT>(prm, f, g, c, dx, dy, lap, D.step2 != 0 && next_to_solid,
                       D.step2_relax_j != 0, fo, go);
}

// One time step of the tile at (x0, y0): phi of the tile and its halo into
// ph, then the tile's fluid and wall nodes.  Every thread of the CTA calls it
// (it holds CTA barriers); threads without a node of their own only help
// with phi.
template <typename Real, bool MRT, bool L2ONLY>
__device__ __forceinline__ void geo_tile_step(const DomDesc& D, int parity, int x0, int y0,
                                              const GeoTables& t, Real (&ph)[kGPY][kGPX])
{
    const int nx = D.nx, ny = D.ny;
    const Real* fs = static_cast<const Real*>(parity ? D.f[1] : D.f[0]);
    const Real* gs = static_cast<const Real*>(parity ? D.g[1] : D.g[0]);
    // lattice coordinates (unwrapped, within the halos) to shared memory
    auto cls_l = [&](int x, int y) -> int { return t.cl[y - y0 + kGC][x - x0 + kGC]; };
    // a population pulled from a solid node bounces back (wall nodes stream)
    auto solid_l = [&](int x, int y) {
        const int c = cls_l(x, y);
        return c != 0 && c != kNodeWall;
    };
    auto phi_l = [&](int x, int y) -> Real { return ph[y - y0 + kGH][x - x0 + kGH]; };
    auto off_l = [&](int x, int y) -> int { return t.rowo[y - y0 + kGC] + t.colx[x - x0 + kGC]; };
    // the nine pulled values of fluid node (x, y) from population set src;
    // a solid source bounces back (the node's own reversed population)
    const long long P = D.plane;
    auto pull = [&](const Real* src, int x, int y, Real (&v)[9]) {
        const int own = off_l(x, y);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sx = x - gex(i), sy = y - gey(i);
            if (i != 0 && solid_l(sx, sy))
                v[i] = geo_ld<L2ONLY>(src + gopp(i) * P + own);
            else
                v[i] = geo_ld<L2ONLY>(src + i * P + off_l(sx, sy));
        }
    };
    const int x = x0 + int(threadIdx.x) % kGTX, y = y0 + int(threadIdx.x) / kGTX;
    const int cme = (x < nx && y < ny) ? cls_l(x, y) : 1;
    const bool live = cme == 0 || cme == kNodeWall;
    Real f[9];
    if (live) pull(fs, x, y, f);
    // 2. phi of the tile and its halo (solid nodes: unused); a fixed trip
    // count lets the loads of all of a thread's positions be in flight at once
    constexpr int kPhiIters = (kGPX * kGPY + kGTX * kGTY - 1) / (kGTX * kGTY);
#pragma unroll
    for (int it = 0; it < kPhiIters; ++it) {
        const int k = int(threadIdx.x) + it * kGTX * kGTY;
        if (k >= kGPX * kGPY) break;
        const int py = k / kGPX, px = k - py * kGPX;
        const int hx = x0 - kGH + px, hy = y0 - kGH + py;
        Real v = Real(0);
        if (cls_l(hx, hy) == 0) {
            Real g[9];
            pull(gs, hx, hy, g);
            v = phi_sum<Real>(g);
        }
        ph[py][px] = v;
    }
    __syncthreads();
    // 3. the tile's fluid and wall nodes
    if (!live) return;
    Real* fd = static_cast<Real*>(parity ? D.f[0] : D.f[1]);
    Real* gd = static_cast<Real*>(parity ? D.g[0] : D.g[1]);
    const int o = off_l(x, y);
    Real g[9], fo[9], go[9];
    pull(gs, x, y, g);
    geo_node_update<Real, MRT>(D, x, y, cme, f, g, cls_l, phi_l, fo, go);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        fd[i * P + o] = fo[i];
        gd[i * P + o] = go[i];
    }
}

// Programmatic dependent launch of the per-step kernel: once every CTA of
// one step's grid has started, the next step's grid (launched with
// programmatic stream serialisation) may be scheduled; its CTAs build their
// tables from the static class map, then wait until the previous grid has
// finished and its writes are visible before they touch the state.  The
// next launch and its set-up so overlap the tail of this one.
__device__ __forceinline__ void pdl_allow_next()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename Real, bool MRT>
__global__ void __launch_bounds__(kGTX * kGTY) geo_step_kernel(DomDesc D, int parity)
{
    __shared__ GeoTables t;
    __shared__ Real ph[kGPY][kGPX];
    const int x0 = blockIdx.x * kGTX, y0 = blockIdx.y * kGTY;
    pdl_allow_next();
    geo_tile_setup(D, x0, y0, t);
    pdl_wait_prev();
    geo_tile_step<Real, MRT, false>(D, parity, x0, y0, t, ph);
}

// Two steps per launch (temporal blocking; the state stays in L2, so a step
// is bound by latency, and a launch costs about as much as a step): a CTA
// computes step t on its tile and a kFH-node halo into shared memory, then
// step t + 1 on the tile from there.  Step t + 1 pulls one node beyond the
// tile and takes phi three nodes beyond it, whose g pulls reach one more:
// kFH = 4.  Step t then needs phi of the state at t kFH + kGH nodes beyond
// the tile and the class map one node further.  Halo nodes are computed by
// several CTAs with the same arithmetic (geo_node_update), so the result is
// bit-identical to two single steps.  Reads buffer `parity` and writes the
// other one, which therefore holds step t + 2: the launch flips the handle's
// buffer once.
constexpr int kFH = 4;            // step-t output halo
constexpr int kFP = kFH + kGH;    // phi halo of the state at t
constexpr int kFC = kFP + 1;      // class-map halo
constexpr int kFCX = kGTX + 2 * kFC, kFCY = kGTY + 2 * kFC;
constexpr int kFPX = kGTX + 2 * kFP, kFPY = kGTY + 2 * kFP;
constexpr int kFAX = kGTX + 2 * kFH, kFAY = kGTY + 2 * kFH;

template <typename Real>
struct GeoFused {
    Real fa[9][kFAY][kFAX];  // step-t output on the tile and its kFH halo
    Real ga[9][kFAY][kFAX];
    Real ph0[kFPY][kFPX];    // phi of the state at t
    Real ph1[kGPY][kGPX];    // phi of the state at t + 1
    int colx[kFCX];
    int rowo[kFCY];
    int rowc[kFCY];
    signed char cl[kFCY][kFCX];
};

template <typename Real, bool MRT>
__global__ void __launch_bounds__(kGTX * kGTY) geo_step2_kernel(DomDesc D, int parity)
{
    extern __shared__ __align__(16) unsigned char geo_smem[];
    GeoFused<Real>& S = *reinterpret_cast<GeoFused<Real>*>(geo_smem);
    const int x0 = blockIdx.x * kGTX, y0 = blockIdx.y * kGTY;
    const int nx = D.nx, ny = D.ny;
    const int tid = int(threadIdx.x), nthr = int(blockDim.x);
    // 0. wrapped halo coordinates and the class map on the tile + kFC
    for (int k = tid; k < kFCX + kFCY; k += nthr) {
        if (k < kFCX)
            S.colx[k] = wrap_any(x0 - kFC + k, nx) + kXOff;
        else {
            const int wy = wrap_any(y0 - kFC + (k - kFCX), ny);
            S.rowo[k - kFCX] = wy * D.pitch;
            S.rowc[k - kFCX] = wy * nx;
        }
    }
    __syncthreads();
    for (int k = tid; k < kFCX * kFCY; k += nthr) {
        const int cy = k / kFCX, cx = k - cy * kFCX;
        const int y = y0 - kFC + cy;
        int c;
        if (D.walls && y < 0)
            c = -1;
        else if (D.walls && y >= ny)
            c = -2;
        else
            c = D.cls[S.rowc[cy] + (S.colx[cx] - kXOff)];
        S.cl[cy][cx] = static_cast<signed char>(c);
    }
    __syncthreads();
    auto cls_l = [&](int x, int y) -> int { return S.cl[y - y0 + kFC][x - x0 + kFC]; };
    auto solid_l = [&](int x, int y) {
        const int c = cls_l(x, y);
        return c != 0 && c != kNodeWall;
    };
    auto off_l = [&](int x, int y) -> int { return S.rowo[y - y0 + kFC] + S.colx[x - x0 + kFC]; };
    const long long P = D.plane;
    const Real* fs = static_cast<const Real*>(parity ? D.f[1] : D.f[0]);
    const Real* gs = static_cast<const Real*>(parity ? D.g[1] : D.g[0]);
    // pulls from the state at t (global) and at t + 1 (shared); a solid
    // source bounces back (the node's own reversed population)
    auto pull_g = [&](const Real* src, int x, int y, Real (&v)[9]) {
        const int own = off_l(x, y);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sx = x - gex(i), sy = y - gey(i);
            v[i] = (i != 0 && solid_l(sx, sy)) ? src[gopp(i) * P + own] : src[i * P + off_l(sx, sy)];
        }
    };
    auto pull_s = [&](const Real (&a)[9][kFAY][kFAX], int x, int y, Real (&v)[9]) {
        const int ax = x - x0 + kFH, ay = y - y0 + kFH;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sx = x - gex(i), sy = y - gey(i);
            v[i] = (i != 0 && solid_l(sx, sy)) ? a[gopp(i)][ay][ax]
                                               : a[i][sy - y0 + kFH][sx - x0 + kFH];
        }
    };
    // 1. phi of the state at t on the tile + kFP (fixed trip counts: the
    // loads of all of a thread's positions can be in flight at once)
    constexpr int kT = kGTX * kGTY;
#pragma unroll
    for (int it = 0; it < (kFPX * kFPY + kT - 1) / kT; ++it) {
        const int k = tid + it * kT;
        if (k >= kFPX * kFPY) break;
        const int py = k / kFPX, px = k - py * kFPX;
        const int x = x0 - kFP + px, y = y0 - kFP + py;
        Real v = Real(0);
        if (cls_l(x, y) == 0) {
            Real g[9];
            pull_g(gs, x, y, g);
            v = phi_sum<Real>(g);
        }
        S.ph0[py][px] = v;
    }
    __syncthreads();
    auto phi0_l = [&](int x, int y) -> Real { return S.ph0[y - y0 + kFP][x - x0 + kFP]; };
    // 2. step t on the tile + kFH, into shared memory (solid nodes: unused)
#pragma unroll
    for (int it = 0; it < (kFAX * kFAY + kT - 1) / kT; ++it) {
        const int k = tid + it * kT;
        if (k >= kFAX * kFAY) break;
        const int ay = k / kFAX, ax = k - ay * kFAX;
        const int x = x0 - kFH + ax, y = y0 - kFH + ay;
        const int cme = cls_l(x, y);
        if (cme != 0 && cme != kNodeWall) continue;
        Real f[9], g[9], fo[9], go[9];
        pull_g(fs, x, y, f);
        pull_g(gs, x, y, g);
        geo_node_update<Real, MRT>(D, x, y, cme, f, g, cls_l, phi0_l, fo, go);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            S.fa[i][ay][ax] = fo[i];
            S.ga[i][ay][ax] = go[i];
        }
    }
    __syncthreads();
    // 3. phi of the state at t + 1 on the tile + kGH
#pragma unroll
    for (int it = 0; it < (kGPX * kGPY + kT - 1) / kT; ++it) {
        const int k = tid + it * kT;
        if (k >= kGPX * kGPY) break;
        const int py = k / kGPX, px = k - py * kGPX;
        const int x = x0 - kGH + px, y = y0 - kGH + py;
        Real v = Real(0);
        if (cls_l(x, y) == 0) {
            Real g[9];
            pull_s(S.ga, x, y, g);
            v = phi_sum<Real>(g);
        }
        S.ph1[py][px] = v;
    }
    __syncthreads();
    auto phi1_l = [&](int x, int y) -> Real { return S.ph1[y - y0 + kGH][x - x0 + kGH]; };
    // 4. step t + 1 on the tile, to the other buffer
    const int x = x0 + tid % kGTX, y = y0 + tid / kGTX;
    if (x >= nx || y >= ny) return;
    const int cme = cls_l(x, y);
    if (cme != 0 && cme != kNodeWall) return;
    Real f[9], g[9], fo[9], go[9];
    pull_s(S.fa, x, y, f);
    pull_s(S.ga, x, y, g);
    geo_node_update<Real, MRT>(D, x, y, cme, f, g, cls_l, phi1_l, fo, go);
    Real* fd = static_cast<Real*>(parity ? D.f[0] : D.f[1]);
    Real* gd = static_cast<Real*>(parity ? D.g[0] : D.g[1]);
    const int o = off_l(x, y);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        fd[i * P + o] = fo[i];
        gd[i * P + o] = go[i];
    }
}

// Persistent multi-step form: a cooperative launch (every tile's CTA
// resident at once) runs n_steps steps, one tile per CTA, step s reading
// buffer parity0 ^ (s & flip).  Instead of a launch boundary per step, a tile
// waits before step s until the tiles under its halo (kGC nodes around it,
// periodic; usually its eight neighbours) have finished step s - 1: once
// they are done with step s - 1 they are also done reading what step s
// overwrites (the halo relation is symmetric).  A tile publishes its steps in
// flags[tile] (steps done in this launch) after a CTA barrier and a fence;
// neighbour data is read from L2 (the state changes within the launch).
// The waits are bounded (flag_wait); a give-up stops the CTA at the next
// step.  done[0] counts finished CTAs; the last one resets it and the flags.
// (FP32: four CTAs per SM, so that a 1000 x 120 capillary's 480 tiles are
// resident at once on 152 SMs.)
template <typename Real, bool MRT>
__global__ void __launch_bounds__(kGTX * kGTY, sizeof(Real) == 4 ? 4 : 2)
    geo_persist_kernel(DomDesc D, int parity0, int flip, int n_steps, int* flags, int* done)
{
    __shared__ GeoTables t;
    __shared__ Real ph[kGPY][kGPX];
    __shared__ int nbr[16];
    __shared__ int n_nbr, stop, last_cta;
    const int ntx = int(gridDim.x), nty = int(gridDim.y);
    const int tx = int(blockIdx.x), ty = int(blockIdx.y), me = ty * ntx + tx;
    const int x0 = tx * kGTX, y0 = ty * kGTY;
    geo_tile_setup(D, x0, y0, t);
    if (threadIdx.x == 0) {
        // the tiles under the halo (the wrapped columns and rows of the
        // tables; a short last tile can bring a second tile within reach)
        int cx[4], cy[4], ncx = 0, ncy = 0;
        for (int k = 0; k < kGCX; ++k) {
            const int q = (t.colx[k] - kXOff) / kGTX;
            bool seen = false;
            for (int j = 0; j < ncx; ++j) seen = seen || cx[j] == q;
            if (!seen) cx[ncx++] = q;
        }
        for (int k = 0; k < kGCY; ++k) {
            const int y = y0 - kGC + k;
            if (D.walls && (y < 0 || y >= D.ny)) continue;  // wall rows: no data
            const int q = t.rowc[k] / D.nx / kGTY;
            bool seen = false;
            for (int j = 0; j < ncy; ++j) seen = seen || cy[j] == q;
            if (!seen) cy[ncy++] = q;
        }
        int n = 0;
        for (int a = 0; a < ncy; ++a)
            for (int b = 0; b < ncx; ++b) {
                const int q = cy[a] * ntx + cx[b];
                if (q != me) nbr[n++] = q;
            }
        n_nbr = n;
        stop = 0;
    }
    __syncthreads();
    for (int s = 0; s < n_steps; ++s) {
        if (s > 0) {
            if (int(threadIdx.x) < n_nbr && !flag_wait(flags + nbr[threadIdx.x], s, D.err)) stop = 1;
            __syncthreads();
            if (stop) break;
        }
        geo_tile_step<Real, MRT, true>(D, parity0 ^ (s & flip), x0, y0, t, ph);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_gpu(flags + me, s + 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last_cta = atomicAdd(done, 1) == ntx * nty - 1;
    }
    __syncthreads();
    if (last_cta) {
        __threadfence();
        for (int k = int(threadIdx.x); k < ntx * nty; k += int(blockDim.x)) flags[k] = 0;
        if (threadIdx.x == 0) done[0] = 0;
        __threadfence();
    }
}

// Initial equilibrium (f = f^eq, g = g^eq of phi0 with rho = 1, u = 0) on
// a domain with obstacles; phi0 in FP64 with row pitch D.pitch.  Solid nodes
// get the rest state.  Reads phi0 only at fluid nodes.
template <typename Real>
__global__ void geo_init_eq_kernel(DomDesc D, const double* __restrict__ phi0, int parity)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= D.nx) return;
    Real* fd = static_cast<Real*>(parity ? D.f[1] : D.f[0]);
    Real* gd = static_cast<Real*>(parity ? D.g[1] : D.g[0]);
    const long long P = D.plane;
    const long long o = (long long)y * D.pitch + x + kXOff;
    const GeoView G{D.cls, D.nx, D.ny, D.walls};
    double fe[9], ge[9];
    const int cme = D.cls[(long long)y * D.nx + x];
    if (cme == kNodeWall) {
        // the rest equilibrium of the wall node's wetting phi value
        const int in = y == 0 ? 1 : D.ny - 2;
        const double pw = phi0[(long long)in * D.pitch + x] - (y == 0 ? D.h_bot : D.h_top);
        NodeParams<double> prm{D.a, D.kappa, D.gamma, D.omega_phi, D.tau_c0, D.tau_c1, D.h_bot, D.h_top};
        double m7, m8;
        equilibria<double>(prm, 0.0, pw, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, fe, ge, m7, m8);
        fe[0] = -((((fe[1] + fe[2]) + (fe[3] + fe[4])) + ((fe[5] + fe[6]) + (fe[7] + fe[8]))));
        ge[0] = pw - ((((ge[1] + ge[2]) + (ge[3] + ge[4])) + ((ge[5] + ge[6]) + (ge[7] + ge[8]))));
    } else if (cme != 0) {
        for (int i = 0; i < 9; ++i) fe[i] = ge[i] = 0.0;
    } else {
        // phi0 is laid out with pitch D.pitch; wrap it into a compact view
        auto at = [&](int qx, int qy) -> double {
            return phi0[(long long)wrap_near(qy, D.ny) * D.pitch + wrap_near(qx, D.nx)];
        };
        auto ghost = [&](int qx, int qy) -> double {
            const int k = G.cls_at(qx, qy);
            const double h = k == -1 ? D.h_bot : (k == -2 ? D.h_top : D.hcls[k]);
            double sum = 0.0;
            int n = 0;
            for (int j = 0; j < 4; ++j) {
                const int ddx = j == 0 ? 1 : (j == 1 ? -1 : 0);
                const int ddy = j == 2 ? 1 : (j == 3 ? -1 : 0);
                if (!G.solid(qx + ddx, qy + ddy)) {
                    sum += at(qx + D.wet_k * ddx, qy + D.wet_k * ddy);
                    ++n;
                }
            }
            if (n == 0)
                for (int j = 0; j < 4; ++j) {
                    const int ddx = (j == 0 || j == 3) ? 1 : -1;
                    const int ddy = (j == 0 || j == 2) ? 1 : -1;
                    if (!G.solid(qx + ddx, qy + ddy)) {
                        sum += at(qx + D.wet_k * ddx, qy + D.wet_k * ddy);
                        ++n;
                    }
                }
            const double mean = n == 1 ? sum : (n == 2 ? sum * 0.5 : (n == 3 ? div_const<3>(sum) : sum * 0.25));
            return mean - D.wet_k * h;
        };
        double nb[9];
        for (int i = 1; i < 9; ++i) {
            const int qx = x + gex(i), qy = y + gey(i);
            if (qy >= 0 && qy < D.ny && G.cls_at(qx, qy) == kNodeWall)
                nb[i] = qy == 0 ? at(qx, 1) - D.h_bot : at(qx, D.ny - 2) - D.h_top;
            else
                nb[i] = G.solid(qx, qy) ? ghost(qx, qy) : at(qx, qy);
        }
        const double c = at(x, y);
        double dx, dy, lap, m7, m8;
        stencils<double>(c, nb[1], nb[2], nb[3], nb[4], nb[5], nb[7], nb[8], nb[6], dx, dy, lap);
        NodeParams<double> prm{D.a, D.kappa, D.gamma, D.omega_phi, D.tau_c0, D.tau_c1, D.h_bot, D.h_top};
        equilibria<double>(prm, 0.0, c, 0.0, 0.0, 0.0, 0.0, dx, dy, lap, fe, ge, m7, m8);
        fe[0] = -((((fe[1] + fe[2]) + (fe[3] + fe[4])) + ((fe[5] + fe[6]) + (fe[7] + fe[8]))));
        ge[0] = c - ((((ge[1] + ge[2]) + (ge[3] + ge[4])) + ((ge[5] + ge[6]) + (ge[7] + ge[8]))));
    }
    for (int i = 0; i < 9; ++i) {
        fd[i * P + o] = Real(fe[i]);
        gd[i * P + o] = i == 0 ? G0<Real>::encode(ge[0]) : Real(ge[i]);
    }
}

// Rest state at the solid nodes of buffer b.
template <typename Real>
__global__ void geo_solid_rest_kernel(DomDesc D, int b)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= D.nx || D.cls[(long long)y * D.nx + x] == 0) return;
    Real* fd = static_cast<Real*>(b ? D.f[1] : D.f[0]);
    Real* gd = static_cast<Real*>(b ? D.g[1] : D.g[0]);
    const long long P = D.plane;
    const long long o = (long long)y * D.pitch + x + kXOff;
    for (int i = 0; i < 9; ++i) {
        fd[i * P + o] = Real(0);
        gd[i * P + o] = i == 0 ? G0<Real>::encode(0.0) : Real(0);
    }
}

dim3 geo_grid(const DomDesc& d) { return dim3((d.nx + kGeoBlock - 1) / kGeoBlock, d.ny); }

template <typename Real, bool MRT>
cudaError_t geo_step_t(const DomDesc& d, int parity, cudaStream_t s)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((d.nx + kGTX - 1) / kGTX, (d.ny + kGTY - 1) / kGTY);
    cfg.blockDim = dim3(kGTX * kGTY);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, geo_step_kernel<Real, MRT>, d, parity);
}

template <typename Real, bool MRT>
cudaError_t geo_step2_t(const DomDesc& d, int parity, cudaStream_t s)
{
    const dim3 grid((d.nx + kGTX - 1) / kGTX, (d.ny + kGTY - 1) / kGTY);
    geo_step2_kernel<Real, MRT><<<grid, kGTX * kGTY, sizeof(GeoFused<Real>), s>>>(d, parity);
    return cudaGetLastError();
}

template <typename Real, bool MRT>
cudaError_t geo_step2_prepare()
{
    return cudaFuncSetAttribute(geo_step2_kernel<Real, MRT>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(sizeof(GeoFused<Real>)));
}

template <typename Real, bool MRT>
cudaError_t geo_persist_t(const DomDesc& d, int parity0, int flip, int n_steps, int* flags,
                          int* done, cudaStream_t s)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((d.nx + kGTX - 1) / kGTX, (d.ny + kGTY - 1) / kGTY);
    cfg.blockDim = dim3(kGTX * kGTY);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, geo_persist_kernel<Real, MRT>, d, parity0, flip, n_steps, flags,
                              done);
}

template <typename Real, bool MRT>
int geo_persist_occupancy_t()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, geo_persist_kernel<Real, MRT>, kGTX * kGTY,
                                                      0) != cudaSuccess)
        return 0;
    return n;
}

}  // namespace

int geo_tiles(int nx, int ny) { return ((nx + kGTX - 1) / kGTX) * ((ny + kGTY - 1) / kGTY); }

int geo_persist_occupancy(int precision, int coll)
{
    if (precision == 0)
        return coll ? geo_persist_occupancy_t<float, true>() : geo_persist_occupancy_t<float, false>();
    return coll ? geo_persist_occupancy_t<double, true>() : geo_persist_occupancy_t<double, false>();
}

int launch_geo_persist(int precision, int coll, const DomDesc& d, int parity0, int flip,
                       int n_steps, int* flags, int* done, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n_steps <= 0) return int(cudaErrorInvalidValue);
    if (precision == 0)
        return int(coll ? geo_persist_t<float, true>(d, parity0, flip, n_steps, flags, done, s)
                        : geo_persist_t<float, false>(d, parity0, flip, n_steps, flags, done, s));
    return int(coll ? geo_persist_t<double, true>(d, parity0, flip, n_steps, flags, done, s)
                    : geo_persist_t<double, false>(d, parity0, flip, n_steps, flags, done, s));
}

int launch_geo_step2(int precision, int coll, const DomDesc& d, int parity, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == 0)
        return int(coll ? geo_step2_t<float, true>(d, parity, s) : geo_step2_t<float, false>(d, parity, s));
    return int(coll ? geo_step2_t<double, true>(d, parity, s) : geo_step2_t<double, false>(d, parity, s));
}

int prepare_geo_step2()
{
    const cudaError_t r[] = {geo_step2_prepare<float, false>(), geo_step2_prepare<float, true>(),
                             geo_step2_prepare<double, false>(), geo_step2_prepare<double, true>()};
    for (cudaError_t v : r)
        if (v != cudaSuccess) return int(v);
    return 0;
}

int launch_geo_step(int precision, int coll, const DomDesc& d, int parity, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == 0)
        return int(coll ? geo_step_t<float, true>(d, parity, s) : geo_step_t<float, false>(d, parity, s));
    return int(coll ? geo_step_t<double, true>(d, parity, s) : geo_step_t<double, false>(d, parity, s));
}

int launch_geo_init_eq(int precision, const DomDesc& d, const double* phi0, int parity, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == 0)
        geo_init_eq_kernel<float><<<geo_grid(d), kGeoBlock, 0, s>>>(d, phi0, parity);
    else
        geo_init_eq_kernel<double><<<geo_grid(d), kGeoBlock, 0, s>>>(d, phi0, parity);
    return int(cudaGetLastError());
}

int launch_geo_solid_rest(int precision, const DomDesc& d, int b, void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == 0)
        geo_solid_rest_kernel<float><<<geo_grid(d), kGeoBlock, 0, s>>>(d, b);
    else
        geo_solid_rest_kernel<double><<<geo_grid(d), kGeoBlock, 0, s>>>(d, b);
    return int(cudaGetLastError());
}

}  // namespace lbfe
