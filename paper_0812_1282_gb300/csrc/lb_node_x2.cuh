// The FP32 per-node arithmetic of lb_node.cuh on two nodes at once, with
// the packed FP32 add, multiply and fused multiply-add of sm_100 and later
// (one instruction for both lanes, half the issue slots of the scalar
// form).  Each lane evaluates the same
// formulas as the scalar path for its own node (Appendix A equilibria,
// Eq. best stencils, Eq. chempot, Eq. tau, Steps 1-3 of Sec. V), with the
// same unbiased divisions by small constants; products that feed a sum are
// fused explicitly, so a lane can differ from the scalar path by rounding.
#pragma once

#include <cuda_runtime.h>

#include "lb_node.cuh"

namespace lbfe {

// Two FP32 lanes.
struct f2 {
    float2 v;
    __device__ __forceinline__ f2() {}
    __device__ __forceinline__ f2(float2 a) : v(a) {}
    __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit f2(float a) : v(make_float2(a, a)) {}
    __device__ __forceinline__ float lane(int l) const { return l ? v.y : v.x; }
};
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
// a - b, one rounding (the product with -1 is exact)
__device__ __forceinline__ f2 operator-(f2 a, f2 b)
{
    return f2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v));
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator*(float k, f2 b)
{
    return f2(__fmul2_rn(make_float2(k, k), b.v));
}
// a * b + c, one rounding
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ f2 fma2(float k, f2 b, f2 c)
{
    return f2(__ffma2_rn(make_float2(k, k), b.v, c.v));
}

// The node parameters P of the functions below are a NodeParams<float> or a
// volatile one (in shared memory, read at each use).

// x / K, unbiased (the residual step of div_const<K, float>)
template <int K>
__device__ __forceinline__ f2 div_const2(f2 x)
{
    constexpr float r = 1.0f / float(K);
    const f2 q = r * x;
    return fma2(r, fma2(-float(K), q, x), q);
}

// correctly rounded reciprocal, lane by lane (no packed form)
__device__ __forceinline__ f2 rcp2(f2 x) { return f2(__frcp_rn(x.v.x), __frcp_rn(x.v.y)); }

// G0<float>::value / advance lane by lane (integer words)
__device__ __forceinline__ f2 g0_value2(f2 w)
{
    return 0x1p-29f *
           f2(__int2float_rn(__float_as_int(w.v.x)), __int2float_rn(__float_as_int(w.v.y)));
}
__device__ __forceinline__ f2 g0_advance2(f2 w, f2 d)
{
    const f2 s = 0x1p29f * d;
    return f2(__int_as_float(__float_as_int(w.v.x) + __float2int_rn(s.v.x)),
              __int_as_float(__float_as_int(w.v.y) + __float2int_rn(s.v.y)));
}

// Eq. (best) on absolute values, differences to the centre first (exact for
// nearby values, as in stencils<float>)
__device__ __forceinline__ void stencils2(f2 c, f2 e, f2 w, f2 n, f2 s, f2 ne, f2 nw, f2 se,
                                          f2 sw, f2& dx, f2& dy, f2& lap)
{
    const f2 de = e - c, dw = w - c, dn = n - c, ds = s - c;
    const f2 dne = ne - c, dnw = nw - c, dse = se - c, dsw = sw - c;
    dx = div_const2<12>(fma2(4.f, de - dw, dne - dnw) + (dse - dsw));
    dy = div_const2<12>(fma2(4.f, dn - ds, dne - dse) + (dnw - dsw));
    lap = div_const2<6>(fma2(4.f, (de + dw) + (dn + ds), (dne + dnw) + (dse + dsw)));
}

// Appendix A equilibria for i = 1..8 in deviation form (f_equilibria)
template <class PP>
__device__ __forceinline__ void f_equilibria2(PP& P, f2 drho, f2 phi, f2 jxe,
                                              f2 jye, f2 uxe, f2 uye, f2 dx, f2 dy, f2 lap,
                                              f2 (&fe)[9], f2& m7eq, f2& m8eq)
{
    const f2 phi2 = phi * phi;
    // 3 [p0 - kappa phi lap] - rho
    const f2 A3 = fma2(-3.f * P.kappa, phi * lap,
                       fma2(P.a * phi2, fma2(2.25f, phi2, f2(-1.5f)), drho));
    const f2 rxx = jxe * uxe, ryy = jye * uye, rxy = jxe * uye;
    const f2 ruu = rxx + ryy;
    const f2 kdx = P.kappa * dx, kdy = P.kappa * dy;
    const f2 kxx = kdx * dx, kyy = kdy * dy, kxy = kdx * dy;
    const f2 ksum = kxx + kyy;
    m7eq = (rxx - ryy) + (kxx - kyy);
    m8eq = rxy + kxy;
    const f2 A4 = 4.f * A3, r6 = -6.f * ruu;
    const f2 Bx = A4 + fma2(18.f, rxx, r6) + fma2(12.f, kxx, -6.f * kyy);
    const f2 By = A4 + fma2(18.f, ryy, r6) + fma2(12.f, kyy, -6.f * kxx);
    const f2 Bb = fma2(-1.5f, ksum, fma2(3.f, ruu, A3));
    const f2 x9 = 9.f * (rxy + kxy);
    const f2 Bd = Bb + x9, Ba = Bb - x9;
    const f2 jp = jxe + jye, jm = jye - jxe;
    fe[1] = div_const2<36>(fma2(12.f, jxe, Bx));
    fe[2] = div_const2<36>(fma2(-12.f, jxe, Bx));
    fe[3] = div_const2<36>(fma2(12.f, jye, By));
    fe[4] = div_const2<36>(fma2(-12.f, jye, By));
    fe[5] = div_const2<36>(fma2(3.f, jp, Bd));
    fe[6] = div_const2<36>(fma2(-3.f, jp, Bd));
    fe[7] = div_const2<36>(fma2(3.f, jm, Ba));
    fe[8] = div_const2<36>(fma2(-3.f, jm, Ba));
}

// Gamma mu, Eq. (chempot)
template <class PP>
__device__ __forceinline__ f2 gamma_mu2(PP& P, f2 phi, f2 lap)
{
    const f2 mu = fma2(-P.kappa, lap, P.a * fma2(phi * phi, phi, f2(0.f) - phi));
    return P.gamma * mu;
}

// g equilibria for i = 1..8 (g_equilibria)
__device__ __forceinline__ void g_equilibria2(f2 phi, f2 G, f2 uxe, f2 uye, f2 (&ge)[9])
{
    const f2 pux = phi * uxe, puy = phi * uye;
    const f2 pxx = pux * uxe, pyy = puy * uye, pxy = pux * uye;
    const f2 puu = pxx + pyy;
    const f2 G4 = 4.f * G, p2 = -2.f * puu;
    const f2 Cx = G4 + fma2(6.f, pxx, p2);
    const f2 Cy = G4 + fma2(6.f, pyy, p2);
    const f2 Gp = G + puu, x3 = 3.f * pxy;
    const f2 Cd = Gp + x3, Ca = Gp - x3;
    const f2 sp = pux + puy, sm = puy - pux;
    ge[1] = div_const2<12>(fma2(4.f, pux, Cx));
    ge[2] = div_const2<12>(fma2(-4.f, pux, Cx));
    ge[3] = div_const2<12>(fma2(4.f, puy, Cy));
    ge[4] = div_const2<12>(fma2(-4.f, puy, Cy));
    ge[5] = div_const2<12>(Cd + sp);
    ge[6] = div_const2<12>(Cd - sp);
    ge[7] = div_const2<12>(Ca + sm);
    ge[8] = div_const2<12>(Ca - sm);
}

__device__ __forceinline__ f2 g_tail_sum2(const f2 (&g)[9])
{
    return (((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8])));
}

// The f part of Steps 1-3 (collide_f) for two nodes of one row.  step2 and
// step2_relax_j are those of the row.
template <bool MRT, class PP>
__device__ __forceinline__ void collide_f2(PP& P, const f2 (&f)[9], f2 phi,
                                           f2 dx, f2 dy, f2 lap, bool step2, bool step2_relax_j,
                                           f2 (&fo)[9], f2& uxe_out, f2& uye_out)
{
    const f2 drho = (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]))) + f[8];
    const f2 jx = (f[1] - f[2]) + (f[5] - f[6]) + (f[8] - f[7]);
    const f2 jy = (f[3] - f[4]) + (f[5] - f[6]) + (f[7] - f[8]);
    const f2 irho = rcp2(f2(1.f) + drho);
    // Eq. (tau), with the lookup table of Sec. V lane by lane
    f2 tau = P.tau_c1 == 0.f ? f2(P.tau_c0) : fma2(P.tau_c1, phi, f2(P.tau_c0));
    if (P.lut_kmax > 0.f) {
        float t2[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const float k =
                fminf(fmaxf(rintf((tau.lane(l) - P.lut_lo) * P.lut_inv), 0.f), P.lut_kmax);
            t2[l] = P.lut_lo + k * P.lut_step;
        }
        tau = f2(t2[0], t2[1]);
    }
    const f2 omega = rcp2(tau);
    // Step 2
    const f2 zero(0.f);
    const f2 jxe = step2 ? zero : jx, jye = step2 ? zero : jy;
    const f2 uxe = step2 ? zero : jx * irho, uye = step2 ? zero : jy * irho;
    f2 fe[9], m7eq, m8eq;
    f_equilibria2(P, drho, phi, jxe, jye, uxe, uye, dx, dy, lap, fe, m7eq, m8eq);
    // Step 3
    if (MRT) {
        const f2 m7 = ((f[1] + f[2]) - (f[3] + f[4])) - m7eq;
        const f2 m8 = ((f[5] + f[6]) - (f[7] + f[8])) - m8eq;
        const f2 s = fma2(-0.25f, omega, f2(0.25f));  // (1 - w) / 4
        const f2 c7 = s * m7, c8 = s * m8;
        fo[1] = fe[1] + c7;
        fo[2] = fe[2] + c7;
        fo[3] = fe[3] - c7;
        fo[4] = fe[4] - c7;
        fo[5] = fe[5] + c8;
        fo[6] = fe[6] + c8;
        fo[7] = fe[7] - c8;
        fo[8] = fe[8] - c8;
        // momentum rows: j - j^eq is zero except on Step-2 rows, where the
        // literal rate 0 keeps it (the alternative reading relaxes it)
        if (step2 && !step2_relax_j) {
            const f2 cx = div_const2<6>(jx), cy = div_const2<6>(jy);
            const f2 cp = cx + cy, cm = cy - cx;
            fo[1] = fo[1] + cx;
            fo[2] = fo[2] - cx;
            fo[3] = fo[3] + cy;
            fo[4] = fo[4] - cy;
            fo[5] = fo[5] + cp;
            fo[6] = fo[6] - cp;
            fo[7] = fo[7] + cm;
            fo[8] = fo[8] - cm;
        }
    } else {
        const f2 k = f2(1.f) - omega;
#pragma unroll
        for (int i = 1; i < 9; ++i) fo[i] = fma2(k, f[i] - fe[i], fe[i]);
    }
    fo[0] = drho - ((((fo[1] + fo[2]) + (fo[3] + fo[4])) + ((fo[5] + fo[6]) + (fo[7] + fo[8]))));
    uxe_out = uxe;
    uye_out = uye;
}

}  // namespace lbfe
