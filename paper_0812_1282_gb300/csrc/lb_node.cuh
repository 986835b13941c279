// Per-node arithmetic of the binary-fluid lattice Boltzmann step, shared by
// the step, initialisation and diagnostic kernels (device code only).
//
// Storage is in deviation form for f: the stored value is f_i - t_i with
// t = (4/9, 1/9 x4, 1/36 x4) the rest-state weights (rho = 1, u = 0), so
// that rho - 1 and rho*u come out of sums of small numbers.  g_1..g_8 are
// stored as is (their rest state is 0).  g_0 carries phi itself (|phi| ~ 1),
// so in FP32 it is stored as a 32-bit fixed-point number with resolution
// 2^-29 (range +-4) and advanced by an exact integer add of its small
// conserved increment; FP64 stores it as a double.  See G0<Real>.  (On
// this GPU integer/float conversions issue on the slow FP64 pipe, so a node
// converts its g_0 word once, when its phi is formed, and once back.)
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

namespace lbfe {

// The node functions below take their parameters P as a NodeParams<Real>
// or as a volatile one (in shared memory, read at each use).
template <typename Real>
struct NodeParams {
    Real a, kappa, gamma, omega_phi, tau_c0, tau_c1, h_bot, h_top;
    Real lut_lo, lut_step, lut_inv, lut_kmax;  // lookup table of Sec. V (kmax 0: off)
};

template <typename Real>
__device__ __forceinline__ Real rcp_rn(Real x);
template <>
__device__ __forceinline__ float rcp_rn<float>(float x) { return __frcp_rn(x); }
template <>
__device__ __forceinline__ double rcp_rn<double>(double x) { return __drcp_rn(x); }

// x / K for a small integer constant K, unbiased.  In FP32 the product with
// the rounded reciprocal fl(1/K) carries a systematic relative bias (e.g.
// +3e-8 for K = 3); one FMA residual step removes it (the result is the
// correctly rounded quotient up to rare ties).  A coherent bias in the
// equilibrium weights or stencil constants acts like a persistent force and
// drives a slow drift of the interface, so every division of the node
// arithmetic goes through here.
template <int K, typename Real>
__device__ __forceinline__ Real div_const(Real x);
template <int K>
__device__ __forceinline__ float div_const(float x)
{
    constexpr float r = 1.0f / float(K);
    const float q = x * r;
    return fmaf(fmaf(-q, float(K), x), r, q);
}
// In FP64 the rounded reciprocal's bias (~1e-16) is far below anything the
// double build is checked at, and an IEEE division costs about fifteen
// instructions on the slow FP64 pipe, so a plain product is used.
template <int K>
__device__ __forceinline__ double div_const(double x)
{
    constexpr double r = 1.0 / double(K);
    return x * r;
}

// Storage of g_0.  value(): the number a stored word represents;
// advance(raw, d): the stored word of value(raw) + d.
template <typename Real>
struct G0;
template <>
struct G0<float> {
    static constexpr double kScale = 536870912.0;  // 2^29
    __device__ __forceinline__ static float value(float raw)
    {
        return __int2float_rn(__float_as_int(raw)) * 0x1p-29f;
    }
    __device__ __forceinline__ static float advance(float raw, float d)
    {
        return __int_as_float(__float_as_int(raw) + __float2int_rn(d * 0x1p29f));
    }
    __host__ __device__ static float encode(double v)
    {
#ifdef __CUDA_ARCH__
        return __int_as_float(__double2int_rn(v * kScale));
#else
        const int i = int(std::nearbyint(v * kScale));
        float f;
        memcpy(&f, &i, sizeof(f));
        return f;
#endif
    }
    __host__ __device__ static double decode(float raw)
    {
#ifdef __CUDA_ARCH__
        return double(__float_as_int(raw)) / kScale;
#else
        int i;
        memcpy(&i, &raw, sizeof(i));
        return double(i) / kScale;
#endif
    }
};
template <>
struct G0<double> {
    __device__ __forceinline__ static double value(double raw) { return raw; }
    __device__ __forceinline__ static double advance(double raw, double d) { return raw + d; }
    __host__ __device__ static double encode(double v) { return v; }
    __host__ __device__ static double decode(double raw) { return raw; }
};

// phi = sum_i g_i (Eq. moments) from stored words, always in this order so
// that every thread that evaluates phi at a node gets the same bits.
template <typename Real>
__device__ __forceinline__ Real phi_sum(const Real (&g)[9])
{
    return (((G0<Real>::value(g[0]) + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]))) +
           g[8];
}

// sum of g_1..g_8
template <typename Real>
__device__ __forceinline__ Real g_tail_sum(const Real (&g)[9])
{
    return (((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8])));
}

// Eq. (best): isotropic gradient (1/12 [-1 0 1; -4 0 4; -1 0 1] and its
// transpose) and nine-point Laplacian (1/6 [1 4 1; 4 -20 4; 1 4 1]),
// written on the differences d* = phi(neighbour) - phi(centre) (the weights
// sum to zero; near a bulk phase the differences of nearby values are exact).
template <typename Real>
__device__ __forceinline__ void stencils_diff(Real e, Real w, Real n, Real s, Real ne, Real nw,
                                              Real se, Real sw, Real& dx, Real& dy, Real& lap)
{
    dx = div_const<12>(Real(4) * (e - w) + (ne - nw) + (se - sw));
    dy = div_const<12>(Real(4) * (n - s) + (ne - se) + (nw - sw));
    lap = div_const<6>(Real(4) * ((e + w) + (n + s)) + ((ne + nw) + (se + sw)));
}

// Same stencils on absolute values.  FP32 forms the differences first
// (exact for nearby values, so a bulk phase's Laplacian carries no
// cancellation error); FP64 needs no such care and uses fewer operations.
template <typename Real>
__device__ __forceinline__ void stencils(Real c, Real e, Real w, Real n, Real s, Real ne, Real nw,
                                         Real se, Real sw, Real& dx, Real& dy, Real& lap);
template <>
__device__ __forceinline__ void stencils<float>(float c, float e, float w, float n, float s,
                                                float ne, float nw, float se, float sw, float& dx,
                                                float& dy, float& lap)
{
    stencils_diff<float>(e - c, w - c, n - c, s - c, ne - c, nw - c, se - c, sw - c, dx, dy, lap);
}
template <>
__device__ __forceinline__ void stencils<double>(double c, double e, double w, double n, double s,
                                                 double ne, double nw, double se, double sw,
                                                 double& dx, double& dy, double& lap)
{
    dx = div_const<12>(4.0 * (e - w) + (ne - nw) + (se - sw));
    dy = div_const<12>(4.0 * (n - s) + (ne - se) + (nw - sw));
    lap = div_const<6>(4.0 * ((e + w) + (n + s)) + ((ne + nw) + (se + sw)) - 20.0 * c);
}

// Equilibria of Appendix A (Eq. equilibrium) for i = 1..8, f in deviation
// form: fe[i] = f^eq_i - t_i, using w_i p0 = t_i rho + w_i a(-phi^2/2 +
// 3 phi^4/4) (Eq. p0, c = 1).  (jxe, jye) = rho u_eq and (uxe, uye) = u_eq
// are the equilibrium momentum / velocity (zero at Step-2 nodes).
// Written as 36 fe_i and 12 ge_i, whose coefficients (the weights w_i,
// w^xx, w^yy, w^xy and the 3/2 of the velocity terms, times 36 or 12) are
// exact, followed by one unbiased division each.
// m7eq / m8eq receive the two stress moments of f^eq (rows 7, 8 of Eq.
// Matrix): (fe1 + fe2) - (fe3 + fe4) = rho(ux^2 - uy^2) + kappa(dx^2 - dy^2) and
// (fe5 + fe6) - (fe7 + fe8) = rho ux uy + kappa dx dy.
template <typename Real, class PP>
__device__ __forceinline__ void f_equilibria(PP& P, Real drho, Real phi,
                                             Real jxe, Real jye, Real uxe, Real uye, Real dx,
                                             Real dy, Real lap, Real (&fe)[9], Real& m7eq,
                                             Real& m8eq)
{
    const Real phi2 = phi * phi;
    // 3 x isotropic part: 3 [p0 - kappa phi lap] - rho (Eq. p0 minus the rest pressure)
    const Real A3 = drho + P.a * phi2 * (Real(2.25) * phi2 - Real(1.5)) -
                    Real(3) * P.kappa * phi * lap;
    // rho u_a u_b
    const Real rxx = jxe * uxe, ryy = jye * uye, rxy = jxe * uye;
    const Real ruu = rxx + ryy;
    // kappa d_a phi d_b phi
    const Real kxx = P.kappa * dx * dx, kyy = P.kappa * dy * dy, kxy = P.kappa * dx * dy;
    const Real ksum = kxx + kyy;
    m7eq = (rxx - ryy) + (kxx - kyy);
    m8eq = rxy + kxy;
    // 36 fe_i = even part + odd (momentum) part
    const Real Bx = Real(4) * A3 + Real(18) * rxx - Real(6) * ruu + Real(12) * kxx - Real(6) * kyy;
    const Real By = Real(4) * A3 + Real(18) * ryy - Real(6) * ruu - Real(6) * kxx + Real(12) * kyy;
    const Real Bd = A3 + Real(3) * ruu + Real(9) * rxy - Real(1.5) * ksum + Real(9) * kxy;  // +-(1,1)
    const Real Ba = A3 + Real(3) * ruu - Real(9) * rxy - Real(1.5) * ksum - Real(9) * kxy;  // +-(-1,1)
    fe[1] = div_const<36>(Bx + Real(12) * jxe);
    fe[2] = div_const<36>(Bx - Real(12) * jxe);
    fe[3] = div_const<36>(By + Real(12) * jye);
    fe[4] = div_const<36>(By - Real(12) * jye);
    fe[5] = div_const<36>(Bd + Real(3) * (jxe + jye));
    fe[6] = div_const<36>(Bd - Real(3) * (jxe + jye));
    fe[7] = div_const<36>(Ba + Real(3) * (jye - jxe));
    fe[8] = div_const<36>(Ba - Real(3) * (jye - jxe));
}

// Gamma mu with the chemical potential of Eq. (chempot).
template <typename Real, class PP>
__device__ __forceinline__ Real gamma_mu(PP& P, Real phi, Real lap)
{
    const Real mu = P.a * (phi * phi * phi - phi) - P.kappa * lap;
    return P.gamma * mu;
}

// g equilibria for i = 1..8 from phi, G = Gamma mu and the equilibrium
// velocity: w_i [G + phi e.u + 3/2 phi (e.u e.u - u.u/3)], times 12.
template <typename Real>
__device__ __forceinline__ void g_equilibria(Real phi, Real G, Real uxe, Real uye, Real (&ge)[9])
{
    const Real pux = phi * uxe, puy = phi * uye;
    const Real pxx = pux * uxe, pyy = puy * uye, pxy = pux * uye;
    const Real puu = pxx + pyy;
    const Real Cx = Real(4) * G + Real(6) * pxx - Real(2) * puu;
    const Real Cy = Real(4) * G + Real(6) * pyy - Real(2) * puu;
    const Real Cd = G + puu + Real(3) * pxy;
    const Real Ca = G + puu - Real(3) * pxy;
    ge[1] = div_const<12>(Cx + Real(4) * pux);
    ge[2] = div_const<12>(Cx - Real(4) * pux);
    ge[3] = div_const<12>(Cy + Real(4) * puy);
    ge[4] = div_const<12>(Cy - Real(4) * puy);
    ge[5] = div_const<12>(Cd + (pux + puy));
    ge[6] = div_const<12>(Cd - (pux + puy));
    ge[7] = div_const<12>(Ca + (puy - pux));
    ge[8] = div_const<12>(Ca - (puy - pux));
}

template <typename Real, class PP>
__device__ __forceinline__ void equilibria(PP& P, Real drho, Real phi,
                                           Real jxe, Real jye, Real uxe, Real uye, Real dx,
                                           Real dy, Real lap, Real (&fe)[9], Real (&ge)[9],
                                           Real& m7eq, Real& m8eq)
{
    f_equilibria<Real>(P, drho, phi, jxe, jye, uxe, uye, dx, dy, lap, fe, m7eq, m8eq);
    g_equilibria<Real>(phi, gamma_mu<Real>(P, phi, lap), uxe, uye, ge);
}

// One node of Steps 1-3 (Sec. V): moments of the pulled populations f, g
// (g[0] a stored word, see G0),
// thermodynamics from the phi stencil values, Step 2, equilibria and BGK
// or MRT collision.  fo, go receive the post-collision populations (f in
// deviation form, go[0] a stored word).  f'_0 and g'_0 follow from
// conservation of rho and phi, which both collisions satisfy exactly
// (Eq. feq0, S_0 = 0): g'_0 = g_0 + (sum_{i>0} g_i - sum_{i>0} g'_i).
//
// MRT: f' = f - M^-1 S M (f - f^eq) with S = diag(0,1,1,0,1,0,1,w,w) is
// evaluated as f' = f^eq + M^-1 (I - S) M (f - f^eq): only the momentum
// rows (rate 0; non-zero only where Step 2 zeroes u_eq) and the two stress
// rows (rate w) survive, so
//   f'_i = f^eq_i + M_3i dj_x/6 + M_5i dj_y/6 + (1-w)(M_7i m_7 + M_8i m_8)/4,
// with m_7 = d1+d2-d3-d4, m_8 = d5+d6-d7-d8, d = f - f^eq.  With
// step2_relax_j the momentum rows of a Step-2 node relax at rate 1 instead
// (the dj terms vanish and the node leaves the collision at rest).
// The f part of Steps 1-3 at one node: returns the post-collision f and,
// for the g update, the equilibrium velocity (zero at Step-2 nodes).
template <typename Real, bool MRT, class PP>
__device__ __forceinline__ void collide_f(PP& P, const Real (&f)[9], Real phi,
                                          Real dx, Real dy, Real lap, bool step2,
                                          bool step2_relax_j, Real (&fo)[9], Real& uxe_out,
                                          Real& uye_out)
{
    // Step 1 (Eq. moments); t_i e_i sums to zero, so deviations give j directly
    const Real drho = (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]))) + f[8];
    const Real jx = (f[1] - f[2]) + (f[5] - f[6]) + (f[8] - f[7]);
    const Real jy = (f[3] - f[4]) + (f[5] - f[6]) + (f[7] - f[8]);
    const Real rho = Real(1) + drho;
    const Real irho = rcp_rn(rho);
    // Eq. (tau); equal phase viscosities give a constant rate; with the lookup
    // table of Sec. V the nearest tabulated tau
    Real tau = P.tau_c1 == Real(0) ? P.tau_c0 : P.tau_c0 + P.tau_c1 * phi;
    if (P.lut_kmax > Real(0)) {
        const Real k = fmin(fmax(rint((tau - P.lut_lo) * P.lut_inv), Real(0)), P.lut_kmax);
        tau = P.lut_lo + k * P.lut_step;
    }
    const Real omega = rcp_rn(tau);
    // Step 2
    Real jxe = jx, jye = jy, uxe = jx * irho, uye = jy * irho;
    if (step2) {
        jxe = Real(0);
        jye = Real(0);
        uxe = Real(0);
        uye = Real(0);
    }
    Real fe[9], m7eq, m8eq;
    f_equilibria<Real>(P, drho, phi, jxe, jye, uxe, uye, dx, dy, lap, fe, m7eq, m8eq);
    // Step 3
    if (MRT) {
        const Real m7 = ((f[1] + f[2]) - (f[3] + f[4])) - m7eq;
        const Real m8 = ((f[5] + f[6]) - (f[7] + f[8])) - m8eq;
        const Real s = (Real(1) - omega) * Real(0.25);
        const Real c7 = s * m7, c8 = s * m8;
        // momentum rows: rate 0 (literal Eq. diag) keeps j - j^eq; the alternative
        // reading relaxes it fully on Step-2 rows
        const bool keep_j = !(step2 && step2_relax_j);
        const Real cx = keep_j ? div_const<6>(jx - jxe) : Real(0);
        const Real cy = keep_j ? div_const<6>(jy - jye) : Real(0);
        fo[1] = fe[1] + c7 + cx;
        fo[2] = fe[2] + c7 - cx;
        fo[3] = fe[3] - c7 + cy;
        fo[4] = fe[4] - c7 - cy;
        fo[5] = fe[5] + c8 + (cx + cy);
        fo[6] = fe[6] + c8 - (cx + cy);
        fo[7] = fe[7] - c8 + (cy - cx);
        fo[8] = fe[8] - c8 - (cy - cx);
    } else {
        const Real k = Real(1) - omega;
#pragma unroll
        for (int i = 1; i < 9; ++i) fo[i] = fe[i] + k * (f[i] - fe[i]);
    }
    fo[0] = drho - ((((fo[1] + fo[2]) + (fo[3] + fo[4])) + ((fo[5] + fo[6]) + (fo[7] + fo[8]))));
    uxe_out = uxe;
    uye_out = uye;
}

template <typename Real, bool MRT, class PP>
__device__ __forceinline__ void collide(PP& P, const Real (&f)[9],
                                        const Real (&g)[9], Real phi, Real dx, Real dy, Real lap,
                                        bool step2, bool step2_relax_j, Real (&fo)[9],
                                        Real (&go)[9])
{
    Real uxe, uye, ge[9];
    collide_f<Real, MRT>(P, f, phi, dx, dy, lap, step2, step2_relax_j, fo, uxe, uye);
    g_equilibria<Real>(phi, gamma_mu<Real>(P, phi, lap), uxe, uye, ge);
    // Eq. (gevo); tau_phi = 1 (Sec. III.B) leaves g' = g^eq
    if (P.omega_phi == Real(1)) {
#pragma unroll
        for (int i = 1; i < 9; ++i) go[i] = ge[i];
    } else {
        const Real kg = Real(1) - P.omega_phi;
#pragma unroll
        for (int i = 1; i < 9; ++i) go[i] = ge[i] + kg * (g[i] - ge[i]);
    }
    go[0] = G0<Real>::advance(g[0], g_tail_sum<Real>(g) - g_tail_sum<Real>(go));
}

}  // namespace lbfe
