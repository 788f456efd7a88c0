// Point evaluation of the four kernels K1..K4 of Eq_K1/Eq_K2 (Section 2.2).
//
// With d = x - y, r = |d|, t = kappa r and E = exp(-t) - 1:
//   K1 = (G0 - Gk)                   = -E / (4 pi r)
//   K2 = eps dGk/dn_y - dG0/dn_y     = (n_y.d) / (4 pi r^3) [eps (1 - c1) - 1]
//   K3 = dG0/dn_x - dGk/dn_x / eps   = -(n_x.d) / (4 pi r^3) [1 - (1 - c1) / eps]
//   K4 = d2(Gk - G0)/dn_x dn_y       = [c3 (n_x.d)(n_y.d) / r^2 - c1 (n_x.n_y)] / (4 pi r^3)
// where c1 = 1 - e^-t (1 + t) and c3 = 3 - e^-t (3 + 3t + t^2) are the screened-minus-
// Coulomb radial factors. Both vanish like t^2/2 as t -> 0; writing them through
// g = E + t = t^2/2 - t^3/6 + ... (a Taylor series for small t, exact arithmetic otherwise)
// keeps the relative error of the differences bounded instead of growing like 1/t^2.
#pragma once

#include <cuda_runtime.h>

template <class R>
struct PbKer;

template <>
struct PbKer<double> {
    static __device__ __forceinline__ double expm1_(double x) { return expm1(x); }
    static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
};
template <>
struct PbKer<float> {
    static __device__ __forceinline__ float expm1_(float x) { return expm1f(x); }
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
};

// g(t) = exp(-t) - 1 + t, and E = exp(-t) - 1.
// FP32: below t = 0.125 both come from the Taylor series of g (terms to t^8, truncation
// below 1e-9 relative), E = g - t; above it from exp directly. The two are evaluated
// branch-free and selected, so a warp never diverges on t.
// FP64: exp(-t) - 1 and E + t lose at most ~1e-16/t and ~1e-16/t^2 relative, which stays far
// below the quadrature error at the separations the singular rules sample.
template <class R>
__device__ __forceinline__ void pb_screen(R t, R& E, R& g);

template <>
__device__ __forceinline__ void pb_screen<float>(float t, float& E, float& g)
{
    float s = -1.0f / 40320.0f;        // -1/8! ... the series of g / t^2
    s = fmaf(s, t, 1.0f / 5040.0f);
    s = fmaf(s, t, -1.0f / 720.0f);
    s = fmaf(s, t, 1.0f / 120.0f);
    s = fmaf(s, t, -1.0f / 24.0f);
    s = fmaf(s, t, 1.0f / 6.0f);
    s = fmaf(s, t, -0.5f);
    // s now holds -(g / t^2) up to the sign convention of the alternating series
    float gs = -s * t * t;
    float ed = __expf(-t) - 1.0f;
    bool small = t < 0.125f;
    g = small ? gs : ed + t;
    E = small ? gs - t : ed;
}

template <>
__device__ __forceinline__ void pb_screen<double>(double t, double& E, double& g)
{
    E = exp(-t) - 1.0;
    g = E + t;
}

// K[0..3] = K1..K4 for d = x - y, target normal n_x, source normal n_y, all scaled by `scale`
// (0 drops a pair without extra products: it multiplies 1 / (4 pi r), which every term carries).
template <class R>
__device__ __forceinline__ void pb_kernels(R dx, R dy, R dz, R nxx, R nxy, R nxz, R nyx, R nyy, R nyz,
                                           R eps, R inv_eps, R kappa, R* K, R scale = R(1))
{
    const R i4pi = R(0.07957747154594767) * scale;  // 1 / (4 pi), scaled
    R r2 = dx * dx + dy * dy + dz * dz;
    R rinv = PbKer<R>::rsqrt_(r2);
    R r = r2 * rinv;
    R t = kappa * r;
    R E, g;
    pb_screen<R>(t, E, g);
    R tE = t * E;
    R c1 = -g - tE;
    R c3 = R(-3) * g - t * t - tE * (R(3) + t);
    R ri = rinv * i4pi;
    R ri3 = ri * rinv * rinv;
    R nxd = nxx * dx + nxy * dy + nxz * dz;
    R nyd = nyx * dx + nyy * dy + nyz * dz;
    R nxny = nxx * nyx + nxy * nyy + nxz * nyz;
    R e1 = R(1) - c1;  // e^-t (1 + t)
    K[0] = -E * ri;
    K[1] = nyd * ri3 * (eps * e1 - R(1));
    K[2] = -nxd * ri3 * (R(1) - e1 * inv_eps);
    K[3] = ri3 * (c3 * nxd * nyd * rinv * rinv - c1 * nxny);
}

// The parts from which K1..K4 of both orderings of a pair are assembled:
//   P[0] = K1, P[1] = K4 (both symmetric in x <-> y),
//   P[2] = dG0/dn_y = (n_y.d)/(4 pi r^3),   P[3] = dGk/dn_y = P[2] e^-t (1 + t),
//   P[4] = -dG0/dn_x = (n_x.d)/(4 pi r^3),  P[5] = -dGk/dn_x = P[4] e^-t (1 + t).
// For (x, y): K2 = eps P[3] - P[2], K3 = -P[4] + P[5] / eps; for (y, x): K2 = P[4] - eps P[5],
// K3 = P[2] - P[3] / eps.
template <class R>
__device__ __forceinline__ void pb_kernel_parts(R dx, R dy, R dz, R nxx, R nxy, R nxz, R nyx, R nyy, R nyz, R kappa,
                                                R* P)
{
    const R i4pi = R(0.07957747154594767);
    R r2 = dx * dx + dy * dy + dz * dz;
    R rinv = PbKer<R>::rsqrt_(r2);
    R r = r2 * rinv;
    R t = kappa * r;
    R E, g;
    pb_screen<R>(t, E, g);
    R tE = t * E;
    R c1 = -g - tE;
    R c3 = R(-3) * g - t * t - tE * (R(3) + t);
    R ri = rinv * i4pi;
    R ri3 = ri * rinv * rinv;
    R nxd = nxx * dx + nxy * dy + nxz * dz;
    R nyd = nyx * dx + nyy * dy + nyz * dz;
    R nxny = nxx * nyx + nxy * nyy + nxz * nyz;
    R e1 = R(1) - c1;
    P[0] = -E * ri;
    P[1] = ri3 * (c3 * nxd * nyd * rinv * rinv - c1 * nxny);
    P[2] = nyd * ri3;
    P[3] = P[2] * e1;
    P[4] = nxd * ri3;
    P[5] = P[4] * e1;
}
