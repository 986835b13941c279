// Fused stream + collide time step (Steps 1-4 of Sec. V, pull form).
//
// A CTA owns a strip of blockDim.x columns and marches up through `rows`
// rows, one lattice node per thread per row.  For each row it
//   1. pulls the 9 g populations of the row above (the look-ahead row)
//      and publishes phi there in a 4-row shared-memory ring (the edge
//      threads also publish the two halo columns), then synchronises once;
//   2. pulls the 9 f populations of its own node, reads the 3x3 phi
//      neighbourhood from the ring (wetting ghost rows outside the walls),
//      collides, and stores 18 post-collision values.
// The g values pulled for the look-ahead row are kept in registers and
// reused as the node's own g one row later, so every stored population is
// read from HBM once per step (tile edges re-read from L2).
//
// Pull rule (Eqs. stream1-2 and mid-link bounce-back): f_i(r) =
// f'_i(r - e_i), or f'_opp(i)(r) when r - e_i is inside a wall.
#pragma once

#include "lb_internal.h"
#include "lb_node.cuh"

namespace lbfe {

template <typename Real>
__device__ __forceinline__ NodeParams<Real> node_params(const DomDesc& D)
{
    NodeParams<Real> P;
    P.a = Real(D.a);
    P.kappa = Real(D.kappa);
    P.gamma = Real(D.gamma);
    P.omega_phi = Real(D.omega_phi);
    P.tau_c0 = Real(D.tau_c0);
    P.tau_c1 = Real(D.tau_c1);
    P.h_bot = Real(D.h_bot);
    P.h_top = Real(D.h_top);
    return P;
}

// Row geometry of node row y.
struct RowGeo {
    int c, m, p;      // element offsets of rows y, y-1, y+1 (periodic wrap)
    bool wlo, whi;    // y-1 / y+1 is inside a wall
};

__device__ __forceinline__ RowGeo row_geo(int y, int ny, int pitch, bool walls)
{
    RowGeo r;
    r.c = y * pitch;
    r.m = (y == 0 ? ny - 1 : y - 1) * pitch;
    r.p = (y + 1 == ny ? 0 : y + 1) * pitch;
    r.wlo = walls && (y == 0);
    r.whi = walls && (y + 1 == ny);
    return r;
}

// Pull the nine populations of node (x, row r) from plane set `src`.
template <typename Real>
__device__ __forceinline__ void pull9(const Real* __restrict__ src, int P, const RowGeo& r, int x,
                                      int xm, int xp, Real (&v)[9])
{
    v[0] = __ldg(src + (0 * P + r.c + x));
    v[1] = __ldg(src + (1 * P + r.c + xm));
    v[2] = __ldg(src + (2 * P + r.c + xp));
    v[3] = __ldg(src + (r.wlo ? 4 * P + r.c + x : 3 * P + r.m + x));
    v[4] = __ldg(src + (r.whi ? 3 * P + r.c + x : 4 * P + r.p + x));
    v[5] = __ldg(src + (r.wlo ? 6 * P + r.c + x : 5 * P + r.m + xm));
    v[6] = __ldg(src + (r.whi ? 5 * P + r.c + x : 6 * P + r.p + xp));
    v[7] = __ldg(src + (r.wlo ? 8 * P + r.c + x : 7 * P + r.m + xp));
    v[8] = __ldg(src + (r.whi ? 7 * P + r.c + x : 8 * P + r.p + xm));
}

template <typename Real>
__device__ __forceinline__ PhiRep<Real> pull_phi(const Real* __restrict__ g, int P, const RowGeo& r,
                                                 int x, int xm, int xp)
{
    Real v[9];
    pull9<Real>(g, P, r, x, xm, xp, v);
    return PhiRep<Real>::make(v);
}

template <typename Real, bool MRT>
__device__ __forceinline__ void process_tile(const DomDesc& D, int parity, int x0, int y0, int rows,
                                             PhiRep<Real>* __restrict__ ring)
{
    using Rep = PhiRep<Real>;
    const Real* __restrict__ fs = static_cast<const Real*>((parity ? D.f[1] : D.f[0]));
    const Real* __restrict__ gs = static_cast<const Real*>((parity ? D.g[1] : D.g[0]));
    Real* __restrict__ fd = static_cast<Real*>((parity ? D.f[0] : D.f[1]));
    Real* __restrict__ gd = static_cast<Real*>((parity ? D.g[0] : D.g[1]));
    const int nx = D.nx, ny = D.ny, pitch = D.pitch;
    const int P = static_cast<int>(D.plane);
    const bool walls = D.walls != 0;
    const NodeParams<Real> prm = node_params<Real>(D);

    const int bx = blockDim.x, tx = threadIdx.x, W = bx + 2;
    const int ncols = min(bx, nx - x0);
    const bool active = tx < ncols;
    const int x = x0 + tx;
    const int xm = (x == 0) ? nx - 1 : x - 1;
    const int xp = (x + 1 >= nx) ? 0 : x + 1;
    const bool left = (tx == 0);
    const bool right = (tx == ncols - 1);
    // halo columns and their neighbours (periodic in x)
    const int xl = (x0 == 0) ? nx - 1 : x0 - 1;
    const int xlm = (xl == 0) ? nx - 1 : xl - 1;
    const int xlp = x0;
    const int xr = (x0 + ncols == nx) ? 0 : x0 + ncols;
    const int xrm = x0 + ncols - 1;
    const int xrp = (xr + 1 == nx) ? 0 : xr + 1;
    const int y1 = min(y0 + rows, ny);
    const int own = tx + 1, hr = ncols + 1;

    auto slot = [&](int y) -> Rep* { return ring + ((y - y0 + 1) & 3) * W; };

    // pull g of lattice row y, keep it in gv and publish phi there into the
    // ring slot of row ys (ys = y except across the periodic seam)
    auto publish_row = [&](int y, int ys, Real (&gv)[9]) {
        const RowGeo r = row_geo(y, ny, pitch, walls);
        pull9<Real>(gs, P, r, x, xm, xp, gv);
        Rep* s = slot(ys);
        s[own] = Rep::make(gv);
        if (left) s[0] = pull_phi<Real>(gs, P, r, xl, xlm, xlp);
        if (right) s[hr] = pull_phi<Real>(gs, P, r, xr, xrm, xrp);
    };
    // ghost row yg from the fluid row ys: phi(yg) = phi(ys) - 2h
    auto ghost_row = [&](int yg, int ys, Real h2) {
        Rep* sg = slot(yg);
        const Rep* ss = slot(ys);
        sg[own] = ss[own].minus(h2);
        if (left) sg[0] = ss[0].minus(h2);
        if (right) sg[hr] = ss[hr].minus(h2);
    };

    Real gc[9], gn[9];
    const bool bottom_ghost = walls && (y0 == 0);
    if (active) {
        if (!bottom_ghost) {
            // row y0 - 1 (wraps to ny - 1 only when y is periodic)
            publish_row(y0 == 0 ? ny - 1 : y0 - 1, y0 - 1, gn);
        }
        publish_row(y0, y0, gc);
        if (bottom_ghost) {
            publish_row(1, 1, gn);
            ghost_row(-1, 1, Real(2) * prm.h_bot);
        }
    }
    bool have_next = bottom_ghost;
    for (int y = y0; y < y1; ++y) {
        const int yn = y + 1;
        if (active && !have_next) {
            if (yn < ny) {
                publish_row(yn, yn, gn);
            } else if (walls) {
                ghost_row(yn, ny - 2, Real(2) * prm.h_top);
            } else {
                publish_row(0, yn, gn);  // periodic seam: row 0 sits above row ny - 1
            }
        }
        have_next = false;
        __syncthreads();
        if (active) {
            const RowGeo r = row_geo(y, ny, pitch, walls);
            Real f[9];
            pull9<Real>(fs, P, r, x, xm, xp, f);
            const Rep* sm = slot(y - 1);
            const Rep* sc = slot(y);
            const Rep* sp = slot(y + 1);
            const Rep c = sc[own];
            Real dx, dy, lap;
            stencils_diff<Real>(sc[own + 1] - c, sc[own - 1] - c, sp[own] - c, sm[own] - c,
                                sp[own + 1] - c, sp[own - 1] - c, sm[own + 1] - c,
                                sm[own - 1] - c, dx, dy, lap);
            const bool s2 = D.step2 && (r.wlo || r.whi);
            Real fo[9], go[9];
            collide<Real, MRT>(prm, f, gc, c.value(), dx, dy, lap, s2, fo, go);
            const int o = r.c + x;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                fd[i * P + o] = fo[i];
                gd[i * P + o] = go[i];
            }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) gc[i] = gn[i];
    }
    __syncthreads();  // the ring is reused by the next tile of this CTA
}

}  // namespace lbfe
