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
// A step is two launches on one thread per node: the first forms phi of
// every fluid node from its pulled g (Eq. moments) into a per-node field,
// the second pulls f and g again, takes the phi stencil from that field
// (ghost values at solid neighbours), collides (the node arithmetic of the
// plain step) and stores.  Solid nodes are never written by a step; they
// hold the rest state (f = t, g = 0), so they carry no fluid.
//
// The obstacle path serves small and medium geometries (the capillary set-up
// is ~10^5 nodes), where a step is bound by launch latency rather than by
// HBM bandwidth, so it uses plain coalesced loads instead of the staged
// pipeline of the plain step.
#include <cuda_runtime.h>

#include "lb_internal.h"
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

template <typename Real>
__device__ __forceinline__ Real phi_field(const Real* phi, const GeoView& G, int x, int y)
{
    return phi[(long long)wrap_near(y, G.ny) * G.nx + wrap_near(x, G.nx)];
}

// Wetting ghost value of the solid node (x, y) next to fluid.
template <typename Real>
__device__ Real ghost_phi(const DomDesc& D, const GeoView& G, const Real* phi, int x, int y)
{
    const int k = G.cls_at(x, y);
    const Real h = k == -1 ? (sizeof(Real) == 4 ? Real(D.fh_bot) : Real(D.h_bot))
                 : k == -2 ? (sizeof(Real) == 4 ? Real(D.fh_top) : Real(D.h_top))
                           : class_h<Real>(D, k);
    Real sum = Real(0);
    int n = 0;
    // axis directions (1,0), (-1,0), (0,1), (0,-1)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int dx = j == 0 ? 1 : (j == 1 ? -1 : 0);
        const int dy = j == 2 ? 1 : (j == 3 ? -1 : 0);
        if (!G.solid(x + dx, y + dy)) {
            sum += phi_field(phi, G, x + D.wet_k * dx, y + D.wet_k * dy);
            ++n;
        }
    }
    if (n == 0) {
        // diagonal directions (1,1), (-1,-1), (-1,1), (1,-1)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int dx = (j == 0 || j == 3) ? 1 : -1;
            const int dy = (j == 0 || j == 2) ? 1 : -1;
            if (!G.solid(x + dx, y + dy)) {
                sum += phi_field(phi, G, x + D.wet_k * dx, y + D.wet_k * dy);
                ++n;
            }
        }
    }
    const Real mean = n == 1 ? sum : (n == 2 ? sum * Real(0.5) : (n == 3 ? div_const<3>(sum) : sum * Real(0.25)));
    return mean - Real(D.wet_k) * h;
}

// The nine pulled values of fluid node (x, y) from population set `src`
// (nine planes of D.plane elements, logical column x at x + kXOff).
template <typename Real>
__device__ __forceinline__ void pull9(const DomDesc& D, const GeoView& G, const Real* src, int x,
                                      int y, Real (&v)[9])
{
    const long long P = D.plane;
    const long long own = (long long)y * D.pitch + x + kXOff;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sx = x - gex(i), sy = y - gey(i);
        if (i != 0 && G.solid(sx, sy)) {
            v[i] = src[gopp(i) * P + own];
        } else {
            const long long o = (long long)wrap_near(sy, D.ny) * D.pitch + wrap_near(sx, D.nx) + kXOff;
            v[i] = src[i * P + o];
        }
    }
}

template <typename Real>
__global__ void __launch_bounds__(kGeoBlock) geo_phi_kernel(DomDesc D, int parity)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= D.nx) return;
    const GeoView G{D.cls, D.nx, D.ny, D.walls};
    if (D.cls[(long long)y * D.nx + x] != 0) return;
    const Real* gs = static_cast<const Real*>(parity ? D.g[1] : D.g[0]);
    Real g[9];
    pull9<Real>(D, G, gs, x, y, g);
    static_cast<Real*>(D.phi)[(long long)y * D.nx + x] = phi_sum<Real>(g);
}

template <typename Real, bool MRT>
__global__ void __launch_bounds__(kGeoBlock) geo_step_kernel(DomDesc D, int parity)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= D.nx) return;
    const GeoView G{D.cls, D.nx, D.ny, D.walls};
    if (D.cls[(long long)y * D.nx + x] != 0) return;
    const Real* fs = static_cast<const Real*>(parity ? D.f[1] : D.f[0]);
    const Real* gs = static_cast<const Real*>(parity ? D.g[1] : D.g[0]);
    Real* fd = static_cast<Real*>(parity ? D.f[0] : D.f[1]);
    Real* gd = static_cast<Real*>(parity ? D.g[0] : D.g[1]);
    const Real* phi = static_cast<const Real*>(D.phi);
    Real f[9], g[9];
    pull9<Real>(D, G, fs, x, y, f);
    pull9<Real>(D, G, gs, x, y, g);
    const Real c = phi_sum<Real>(g);
    // phi at the eight neighbours; ghost values at solid ones
    Real nb[9];
    bool next_to_solid = false;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const int qx = x + gex(i), qy = y + gey(i);
        if (G.solid(qx, qy)) {
            next_to_solid = true;
            nb[i] = ghost_phi<Real>(D, G, phi, qx, qy);
        } else {
            nb[i] = phi_field(phi, G, qx, qy);
        }
    }
    Real dx, dy, lap;
    // order: centre, E, W, N, S, NE, NW, SE, SW
    stencils<Real>(c, nb[1], nb[2], nb[3], nb[4], nb[5], nb[7], nb[8], nb[6], dx, dy, lap);
    const NodeParams<Real> prm = geo_params<Real>(D);
    Real fo[9], go[9];
    collide<Real, MRT>(prm, f, g, c, dx, dy, lap, D.step2 != 0 && next_to_solid,
                       D.step2_relax_j != 0, fo, go);
    const long long P = D.plane;
    const long long o = (long long)y * D.pitch + x + kXOff;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        fd[i * P + o] = fo[i];
        gd[i * P + o] = go[i];
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
    if (D.cls[(long long)y * D.nx + x] != 0) {
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
    geo_phi_kernel<Real><<<geo_grid(d), kGeoBlock, 0, s>>>(d, parity);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    geo_step_kernel<Real, MRT><<<geo_grid(d), kGeoBlock, 0, s>>>(d, parity);
    return cudaGetLastError();
}

}  // namespace

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
