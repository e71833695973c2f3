// Host-side tables of a plan, computed in double precision:
//  - the gridding correction S (closed-form Fourier transform of the
//    Kaiser-Bessel kernel),
//  - per-tap polynomial approximations of the kernel for the float path,
//  - FFT twiddle factors,
//  - Daubechies db1..db8 filters by spectral factorisation.
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "host_tables.h"

namespace purify {

static const double kPi = 3.14159265358979323846264338327950288;

// Continuous Fourier transform of g(t) = I0(beta sqrt(1 - (2t/J)^2)) over
// |t| <= J/2 at frequency nu / K:  J sinh(z) / z, z = sqrt(beta^2 - (pi J nu / K)^2),
// continued as J sin(|z|) / |z| for a negative radicand.
double kb_ft(double nu, int J, int K, double beta) {
    double a = beta * beta - (kPi * J * nu / K) * (kPi * J * nu / K);
    if (a > 0) { double z = std::sqrt(a); return J * std::sinh(z) / z; }
    if (a < 0) { double z = std::sqrt(-a); return J * std::sin(z) / z; }
    return (double)J;
}

// s[j] = I0(beta) / ghat(j - n/2): the correction for kernel weights that are
// normalised by I0(beta) (the product over both axes equals 1/(ghat ghat) of
// the unnormalised kernel times the square of that normalisation).
std::vector<double> correction_axis(int n, int K, int J, double beta) {
    std::vector<double> s(n);
    double i0b = bessel_i0_series(beta);
    for (int j = 0; j < n; ++j) s[j] = i0b / kb_ft((double)(j - n / 2), J, K, beta);
    return s;
}

// Chebyshev interpolation of each tap's weight on z = 2 phi - 1 in [-1, 1],
// converted to monomial coefficients for Horner evaluation.
KbPoly fit_kb_poly(int J, double beta, int deg) {
    KbPoly kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.J = J;
    kp.deg = deg;
    const int n = deg + 1;
    double i0b = bessel_i0_series(beta);
    // monomial coefficients of T_0..T_deg
    std::vector<std::vector<double>> T(n, std::vector<double>(n, 0.0));
    T[0][0] = 1.0;
    if (n > 1) T[1][1] = 1.0;
    for (int k = 2; k < n; ++k) {
        for (int i = 0; i < n; ++i) {
            double v = -T[k - 2][i];
            if (i > 0) v += 2.0 * T[k - 1][i - 1];
            T[k][i] = v;
        }
    }
    for (int a = 0; a < J; ++a) {
        std::vector<double> f(n), c(n, 0.0);
        for (int k = 0; k < n; ++k) {
            double z = std::cos(kPi * (k + 0.5) / n);
            double phi = 0.5 * (z + 1.0);
            double t = phi + 0.5 * J - 1.0 - a;
            double r = 1.0 - (2.0 * t / J) * (2.0 * t / J);
            // the kernel is entire in t: continue I0(beta sqrt(r)) by its series in r
            double q = 0.25 * beta * beta * r, term = 1.0, sum = 1.0;
            for (int m = 1; m < 400; ++m) {
                term *= q / ((double)m * (double)m);
                double s2 = sum + term;
                if (s2 == sum && std::fabs(term) < 1e-300 + 1e-18 * std::fabs(sum)) break;
                sum = s2;
            }
            f[k] = sum / i0b;
        }
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int k = 0; k < n; ++k) acc += f[k] * std::cos(kPi * j * (k + 0.5) / n);
            c[j] = acc * 2.0 / n;
        }
        c[0] *= 0.5;
        for (int i = 0; i < n; ++i) {
            double m = 0.0;
            for (int j = 0; j < n; ++j) m += c[j] * T[j][i];
            kp.coef[a][i] = (float)m;
        }
    }
    // the kernel is even in the offset: tap J-1-a at z equals tap a at -z;
    // store the mirrored taps as exact reflections (the middle tap of an odd
    // J as an even polynomial), so that the weights can be evaluated from
    // even and odd parts
    for (int a = 0; a < (J + 1) / 2; ++a)
        for (int i = 0; i < n; ++i) {
            if (2 * a + 1 == J) {
                if (i & 1) kp.coef[a][i] = 0.0f;
            } else {
                kp.coef[J - 1 - a][i] = (i & 1) ? -kp.coef[a][i] : kp.coef[a][i];
            }
        }
    return kp;
}

int kb_poly_degree(int J) { return kb_poly_deg(J); }

std::vector<double> twiddles(int K) {
    // W[t] = exp(-2 pi i t / K) as (re, im) pairs; symmetric evaluation keeps
    // exact zeros and ones at the quarter points
    std::vector<double> w(2 * (size_t)K);
    for (int t = 0; t < K; ++t) {
        int m = t % K;
        double c, s;
        if (4 * m == K) { c = 0.0; s = -1.0; }
        else if (2 * m == K) { c = -1.0; s = 0.0; }
        else if (4 * m == 3 * K) { c = 0.0; s = 1.0; }
        else if (m == 0) { c = 1.0; s = 0.0; }
        else { double ang = 2.0 * kPi * m / K; c = std::cos(ang); s = -std::sin(ang); }
        w[2 * t] = c;
        w[2 * t + 1] = s;
    }
    return w;
}

// Roots of a real polynomial (coefficients lowest degree first) by the
// Durand-Kerner simultaneous iteration in long double complex, then Newton
// polishing on each root.
static std::vector<std::complex<long double>> poly_roots(const std::vector<long double>& c) {
    typedef std::complex<long double> cl;
    int n = (int)c.size() - 1;
    std::vector<cl> r(n);
    if (n <= 0) return r;
    long double lead = c[n];
    auto eval = [&](cl z) {
        cl acc = 0;
        for (int i = n; i >= 0; --i) acc = acc * z + c[i] / lead;
        return acc;
    };
    auto deriv = [&](cl z) {
        cl acc = 0;
        for (int i = n; i >= 1; --i) acc = acc * z + (long double)i * c[i] / lead;
        return acc;
    };
    cl seed(0.4L, 0.9L);
    cl p = 1;
    for (int i = 0; i < n; ++i) { r[i] = p; p *= seed; }
    for (int it = 0; it < 2000; ++it) {
        long double change = 0;
        for (int i = 0; i < n; ++i) {
            cl den = 1;
            for (int j = 0; j < n; ++j) if (j != i) den *= (r[i] - r[j]);
            cl d = eval(r[i]) / den;
            r[i] -= d;
            change = std::max(change, std::abs(d));
        }
        if (change < 1e-30L) break;
    }
    for (int i = 0; i < n; ++i)
        for (int it = 0; it < 5; ++it) {
            cl d = deriv(r[i]);
            if (std::abs(d) == 0) break;
            r[i] -= eval(r[i]) / d;
        }
    return r;
}

// Minimum-phase Daubechies low-pass filter with p vanishing moments (length
// 2p, sum sqrt 2): h is proportional to the polynomial with zeros at -1 (p
// times) and, for each root y_j of P(y) = sum_{k<p} C(p-1+k, k) y^k, the root
// of z^2 - (2 - 4 y_j) z + 1 inside the unit circle; h[0] is the coefficient
// of the highest power.
std::vector<double> daubechies(int p) {
    typedef std::complex<long double> cl;
    std::vector<cl> zeros(p, cl(-1.0L, 0.0L));
    if (p > 1) {
        std::vector<long double> P(p);
        long double binom = 1;  // C(p-1+k, k)
        for (int k = 0; k < p; ++k) {
            if (k > 0) binom = binom * (long double)(p - 1 + k) / (long double)k;
            P[k] = binom;
        }
        for (cl yj : poly_roots(P)) {
            cl c = 1.0L - 2.0L * yj;
            cl d = std::sqrt(c * c - 1.0L);
            cl z1 = c + d, z2 = c - d;
            zeros.push_back(std::abs(z1) < 1.0L ? z1 : z2);
        }
    }
    // expand prod (w - z) with the highest power first
    std::vector<cl> poly(1, cl(1.0L, 0.0L));
    for (cl z : zeros) {
        std::vector<cl> nxt(poly.size() + 1, cl(0, 0));
        for (size_t i = 0; i < poly.size(); ++i) {
            nxt[i] += poly[i];
            nxt[i + 1] -= poly[i] * z;
        }
        poly.swap(nxt);
    }
    long double sum = 0;
    for (cl v : poly) sum += v.real();
    std::vector<double> h(poly.size());
    for (size_t i = 0; i < poly.size(); ++i)
        h[i] = (double)(poly[i].real() * std::sqrt(2.0L) / sum);
    return h;
}

}  // namespace purify
