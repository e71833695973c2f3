// Shared device/host helpers of the imaging library: complex arithmetic,
// the compensated grid-coordinate split used by gridding and by the plan's
// visibility sort, and the Kaiser-Bessel kernel evaluation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define PURIFY_HD __host__ __device__ __forceinline__

namespace purify {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };

// Programmatic dependent launch: wait for the preceding kernel on the stream
// (no-op when the kernel was launched without the attribute), and allow the
// next kernel to be scheduled once this block's work is done.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename C> PURIFY_HD C cmake(decltype(C::x) a, decltype(C::x) b) { C c; c.x = a; c.y = b; return c; }
template <typename C> PURIFY_HD C cadd(C a, C b) { return cmake<C>(a.x + b.x, a.y + b.y); }
template <typename C> PURIFY_HD C csub(C a, C b) { return cmake<C>(a.x - b.x, a.y - b.y); }
template <typename C> PURIFY_HD C cmul(C a, C b) {
    return cmake<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> PURIFY_HD C cmulconj(C a, C b) {  // a * conj(b)
    return cmake<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> PURIFY_HD C cscale(C a, decltype(C::x) s) { return cmake<C>(a.x * s, a.y * s); }

// Largest number of Kaiser-Bessel taps and polynomial coefficients per tap.
#define PURIFY_MAX_J 8
#define PURIFY_MAX_DEG 14

// Grid coordinate constants of one axis: kappa = coord * K / (2 pi), with the
// constant split as c_hi + c_lo in float for a compensated product.
struct AxisConst {
    int K;
    float c_hi, c_lo;
    double c;
};

// Per-tap polynomial approximation of the normalised Kaiser-Bessel kernel:
// tap a at fractional offset phi in [0, 1) has weight
//   g(phi + J/2 - 1 - a) / I0(beta) ~= sum_i coef[a][i] z^i,  z = 2 phi - 1.
struct KbPoly {
    int J, deg;
    float coef[PURIFY_MAX_J][PURIFY_MAX_DEG + 1];
};

// Per-visibility record of the run-ordered gridding work: the fractional
// tap offsets of both axes and the internal visibility index.
struct alignas(16) RunRecF { float phx, phy; int m, pad; };
struct alignas(8) RunRecD { double phx, phy; int m, pad; };
template <typename T> struct RunRecOf;
template <> struct RunRecOf<float> { using type = RunRecF; };
template <> struct RunRecOf<double> { using type = RunRecD; };

// Split kappa = coord * K / (2 pi) into the first tap k0 = floor(kappa - J/2) + 1
// (unwrapped) and phi = (kappa - J/2) - floor(kappa - J/2) in [0, 1), so that
// the tap offsets are t_a = phi + J/2 - 1 - a. Float path: the product is
// compensated (an fma recovers its rounding error, plus the low part of the
// constant), so phi carries the full float precision of the fraction.
PURIFY_HD void split_coord(float coord, const AxisConst& ax, int J, int& k0, float& phi) {
    float p = coord * ax.c_hi;
    float e = fmaf(coord, ax.c_hi, -p);
    e = fmaf(coord, ax.c_lo, e);
    float fl = floorf(p);
    float r = (p - fl) + e;
    if (r < 0.0f) { r += 1.0f; fl -= 1.0f; }
    if (r >= 1.0f) { r -= 1.0f; fl += 1.0f; }
    int ifl = (int)fl;
    if (J & 1) {
        if (r >= 0.5f) { phi = r - 0.5f; k0 = ifl - (J - 1) / 2 + 1; }
        else { phi = r + 0.5f; k0 = ifl - (J - 1) / 2; }
    } else {
        phi = r;
        k0 = ifl - J / 2 + 1;
    }
}

// Double path: kappa in double; floor(kappa - J/2) is exact for J/2 a
// multiple of 1/2 and |kappa| < 2^50.
PURIFY_HD void split_coord(double coord, const AxisConst& ax, int J, int& k0, double& phi) {
    double kappa = coord * ax.c;
    double q = kappa - 0.5 * J;
    double fl = floor(q);
    k0 = (int)fl + 1;
    phi = kappa - (double)k0 - (0.5 * J - 1.0);  // kappa - k0 - (J/2 - 1) = q - fl
}

// Degree of the per-tap polynomial for a J-tap kernel (fixed per J so that
// evaluation unrolls completely): the lowest degree whose Chebyshev
// interpolant of every tap of the normalised kernel (beta = 2.34 J) is within
// 3e-8 of it on [0, 1), below half an FP32 unit at 1.
PURIFY_HD constexpr int kb_poly_deg(int J) { return J <= 3 ? 10 : (J == 4 ? 9 : 8); }

// Float weights of one axis from the per-tap polynomials (Horner in z).
// The kernel is even in the tap offset, so tap J-1-a at z is tap a at -z
// (the host table holds p_{J-1-a}(z) = p_a(-z) exactly): each mirrored pair
// comes from the even and odd parts of p_a, p_a(+-z) = E(z^2) +- z O(z^2),
// Horner in z^2 (the middle tap of an odd J is even).
template <int J>
__device__ __forceinline__ void kb_weights(const KbPoly& kp, float phi, float (&w)[J]) {
    constexpr int DEG = kb_poly_deg(J);
    constexpr int DE = DEG & ~1, DO = (DEG & 1) ? DEG : DEG - 1;   // top even / odd degree
    const float z = fmaf(2.0f, phi, -1.0f);
    const float z2 = z * z;
#pragma unroll
    for (int a = 0; a < (J + 1) / 2; ++a) {
        float e = kp.coef[a][DE];
#pragma unroll
        for (int i = DE - 2; i >= 0; i -= 2) e = fmaf(e, z2, kp.coef[a][i]);
        if (2 * a + 1 == J) {
            w[a] = e;
        } else {
            float o = kp.coef[a][DO];
#pragma unroll
            for (int i = DO - 2; i >= 1; i -= 2) o = fmaf(o, z2, kp.coef[a][i]);
            const float oz = o * z;
            w[a] = e + oz;
            w[J - 1 - a] = e - oz;
        }
    }
}

// Modified Bessel function I0 by its power series sum_k ((x/2)^2)^k / (k!)^2
// (all terms positive; stops once a term no longer changes the sum).
PURIFY_HD double bessel_i0_series(double x) {
    double q = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 200; ++k) {
        term *= q / ((double)k * (double)k);
        double s2 = sum + term;
        if (s2 == sum) break;
        sum = s2;
    }
    return sum;
}

// Double weights of one axis, straight from the kernel definition
// g(t) = I0(beta sqrt(1 - (2t/J)^2)), normalised by I0(beta).
template <int J>
__device__ __forceinline__ void kb_weights(double beta, double inv_i0beta, double phi, double (&w)[J]) {
#pragma unroll
    for (int a = 0; a < J; ++a) {
        double t = phi + (0.5 * J - 1.0 - a);
        double r = 1.0 - (2.0 * t / J) * (2.0 * t / J);
        w[a] = r > 0.0 ? bessel_i0_series(beta * sqrt(r)) * inv_i0beta : (r == 0.0 ? inv_i0beta : 0.0);
    }
}

}  // namespace purify
