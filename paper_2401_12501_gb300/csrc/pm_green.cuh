// Planar Green's function of a~ Delta_2 + c~ for c~ != 0 (Sec. 4.2, eq. diff_param),
// in double precision, callable from host and device code.
//
// With q = c~/a~ real and non-zero, g(r) = a~ G(r; a~, c~) is the Green's function
// of Delta_2 + q, (Delta_2 + q) g = delta:
//
//   q > 0, k = sqrt(q):       g = -(i/4) H0(k r),   H0 = J0 + i Y0 (outgoing);
//   q < 0, kappa = sqrt(-q):  g = -K0(kappa r) / (2 pi)             (decaying).
//
// The sign is the one with unit source strength (2 pi r g'(r) -> 1 as r -> 0), so
// g continues log(r)/(2 pi) of the c~ = 0 case; the paper prints the opposite sign,
// which has source strength -1 under its own small-argument form of H0.
// Radial derivatives, from H0' = -H1, H0'' = -H0 + H1/z, K0' = -K1,
// K1' = -K0 - K1/z:
//
//   q > 0:  g'  = (i k / 4) H1(k r),
//           g'' = (i k^2 / 4) (H0(k r) - H1(k r) / (k r));
//   q < 0:  g'  =  kappa K1(kappa r) / (2 pi),
//           g'' = -kappa^2 (K0(kappa r) + K1(kappa r) / (kappa r)) / (2 pi).
//
// J0, Y0, J1, Y1 are the math library's (j0, y0, j1, y1).  K0 and K1 are
// evaluated here (bessel_k01): the ascending series (Abramowitz & Stegun 9.6.13 and
// 9.6.11 with n = 1) for x <= 2, with t = x^2/4, H_j the harmonic numbers and
// psi(j+1) = -gamma + H_j; above 2 the trapezoid rule on the integral representation
// A&S 9.6.24, whose integrand is analytic in the strip |Im t| < pi/2, so the rule
// converges geometrically.
#pragma once

#include <math.h>

#include <cmath>

namespace pm_green {

constexpr double kPi = 3.14159265358979323846;
constexpr double kEulerGamma = 0.57721566490153286061;

// Coefficients of the float64 series (x <= 2, t = x^2/4 <= 1), computed by the
// compiler from their definitions: c0[j] = 1/(j!)^2, d0[j] = psi(j+1) c0[j],
// c1[j] = 1/(j! (j+1)!), d1[j] = (psi(j+1) + psi(j+2)) c1[j], psi(j+1) = -gamma + H_j.
// Fourteen terms: the last is below 1/(13!)^2 = 2.6e-20 at t = 1.
constexpr int kSeriesK01d = 14;
struct SeriesK01d {
    double c0[kSeriesK01d], d0[kSeriesK01d], c1[kSeriesK01d], d1[kSeriesK01d];
};

__host__ __device__ constexpr SeriesK01d series_k01_d()
{
    SeriesK01d c{};
    double f0 = 1.0, f1 = 1.0, harm = 0.0;      // 1/(j!)^2, 1/(j! (j+1)!), H_j
    for (int j = 0; j < kSeriesK01d; ++j) {
        const double psi1 = -kEulerGamma + harm;
        const double psi2 = psi1 + 1.0 / (j + 1);
        c.c0[j] = f0;
        c.d0[j] = psi1 * f0;
        c.c1[j] = f1;
        c.d1[j] = (psi1 + psi2) * f1;
        harm += 1.0 / (j + 1);
        f0 /= (j + 1.0) * (j + 1.0);
        f1 /= (j + 1.0) * (j + 2.0);
    }
    return c;
}

// Above x = 2, F_nu(x) = sqrt(x) e^x K_nu(x) is smooth in 1/x (it tends to sqrt(pi/2))
// and is expanded in Chebyshev polynomials of z = 4/x - 1 in [-1, 1): 24 terms, whose
// coefficients fall to rounding level by the twentieth.  The coefficients are
// computed once on the host by interpolation at 64 Chebyshev points from reference
// values of F: the trapezoid rule on e^x K_nu(x) = int_0^inf exp(-2 x sinh^2(t/2))
// cosh(nu t) dt (A&S 9.6.24; analytic in the strip |Im t| < pi/2, so geometric
// convergence, step min(1/4, pi^2/(40 + x))) below x = 40, and the asymptotic series
// F_nu ~ sqrt(pi/2) sum_k a_k / x^k, a_k = a_{k-1} (4 nu^2 - (2k - 1)^2)/(8k)
// (A&S 9.7.2) from x = 40, where its smallest term is below 1e-30.  Each translation
// unit that launches kernels evaluating K0/K1 uploads them (upload_cheb_k01).
constexpr int kChebK01 = 24;
struct ChebK01 {
    double c0[kChebK01], c1[kChebK01];
};

inline void scaled_k01_reference(double x, double* F0, double* F1)
{
    if (x >= 40.0) {
        for (int nu = 0; nu < 2; ++nu) {
            double a = 1.0, sum = 1.0;
            for (int k = 1; k < 60; ++k) {
                const double na = a * (4.0 * nu * nu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (8.0 * k * x);
                if (std::fabs(na) >= std::fabs(a) || std::fabs(na) < 1e-30) break;
                a = na;
                sum += a;
            }
            (nu == 0 ? *F0 : *F1) = std::sqrt(0.5 * kPi) * sum;
        }
        return;
    }
    const double h = std::fmin(0.25, kPi * kPi / (40.0 + x));
    double s0 = 0.5, s1 = 0.5;
    for (int j = 1; j <= 400; ++j) {
        const double sh = std::sinh(0.5 * j * h);
        const double e = std::exp(-2.0 * x * sh * sh);
        s0 += e;
        s1 += e * (1.0 + 2.0 * sh * sh);
        if (e < 1e-20 * s0) break;
    }
    *F0 = std::sqrt(x) * h * s0;
    *F1 = std::sqrt(x) * h * s1;
}

inline const ChebK01& cheb_k01_host()
{
    static const ChebK01 table = [] {
        constexpr int M = 64;
        double F0[M], F1[M];
        for (int j = 0; j < M; ++j) {
            const double z = std::cos(kPi * (j + 0.5) / M);
            scaled_k01_reference(4.0 / (z + 1.0), &F0[j], &F1[j]);
        }
        ChebK01 t{};
        for (int k = 0; k < kChebK01; ++k) {
            double a0 = 0.0, a1 = 0.0;
            for (int j = 0; j < M; ++j) {
                const double c = std::cos(k * kPi * (j + 0.5) / M);
                a0 += F0[j] * c;
                a1 += F1[j] * c;
            }
            t.c0[k] = (k == 0 ? 1.0 : 2.0) * a0 / M;
            t.c1[k] = (k == 0 ? 1.0 : 2.0) * a1 / M;
        }
        return t;
    }();
    return table;
}

#ifdef __CUDACC__
static __constant__ ChebK01 g_cheb_k01;      // this translation unit's device copy
static inline cudaError_t upload_cheb_k01()
{
    return cudaMemcpyToSymbol(g_cheb_k01, &cheb_k01_host(), sizeof(ChebK01));
}
#endif

// K0(x), K1(x) for x > 0.
//   x <= 2: K0 = -ln(x/2) I0 + sum_j psi(j+1) t^j/(j!)^2,
//           K1 = 1/x + ln(x/2) I1 - (x/4) sum_j (psi(j+1) + psi(j+2)) t^j/(j! (j+1)!),
//           t = x^2/4 (A&S 9.6.13, 9.6.11), four Horner sums of fourteen terms;
//   x > 2:  K_nu = e^{-x} F_nu(x) / sqrt(x) with F_nu from its Chebyshev expansion
//           (above), summed by Clenshaw's recurrence.
__host__ __device__ inline void bessel_k01(double x, double* k0v, double* k1v)
{
    if (x != x) {                       // NaN passes through (no term count from it)
        *k0v = *k1v = x;
        return;
    }
    if (x <= 2.0) {
        constexpr SeriesK01d C = series_k01_d();
        const double t = 0.25 * x * x;
        double i0 = C.c0[kSeriesK01d - 1], s0 = C.d0[kSeriesK01d - 1];
        double i1s = C.c1[kSeriesK01d - 1], s1 = C.d1[kSeriesK01d - 1];
        for (int j = kSeriesK01d - 2; j >= 0; --j) {
            i0 = fma(i0, t, C.c0[j]);
            s0 = fma(s0, t, C.d0[j]);
            i1s = fma(i1s, t, C.c1[j]);
            s1 = fma(s1, t, C.d1[j]);
        }
        const double lg = log(0.5 * x);
        *k0v = fma(-lg, i0, s0);
        *k1v = 1.0 / x + lg * (0.5 * x * i1s) - 0.25 * x * s1;
        return;
    }
#ifdef __CUDA_ARCH__
    const ChebK01& C = g_cheb_k01;
#else
    const ChebK01& C = cheb_k01_host();
#endif
    const double z = 4.0 / x - 1.0, z2 = 2.0 * z;
    double b01 = 0.0, b02 = 0.0, b11 = 0.0, b12 = 0.0;   // Clenshaw: b_{k+1}, b_{k+2}
    for (int k = kChebK01 - 1; k >= 1; --k) {
        const double t0 = fma(z2, b01, C.c0[k] - b02);
        const double t1 = fma(z2, b11, C.c1[k] - b12);
        b02 = b01;
        b01 = t0;
        b12 = b11;
        b11 = t1;
    }
    const double F0 = fma(z, b01, C.c0[0] - b02), F1 = fma(z, b11, C.c1[0] - b12);
    const double f = exp(-x) / sqrt(x);
    *k0v = F0 * f;
    *k1v = F1 * f;
}

// (g, g', g'') at r > 0 for q = c~/a~ real and non-zero, as (re, im) pairs:
// out[0..1] = g, out[2..3] = g', out[4..5] = g''.
__host__ __device__ inline void green_scaled(double r, double q, double* out)
{
    if (q > 0.0) {
        const double k = sqrt(q);
        const double z = k * r;
        const double J0 = j0(z), Y0 = y0(z), J1 = j1(z), Y1 = y1(z);
        out[0] = 0.25 * Y0;                      // -(i/4)(J0 + i Y0)
        out[1] = -0.25 * J0;
        out[2] = -0.25 * k * Y1;                 // (i k/4)(J1 + i Y1)
        out[3] = 0.25 * k * J1;
        out[4] = -0.25 * k * k * (Y0 - Y1 / z);  // (i k^2/4)(H0 - H1/z)
        out[5] = 0.25 * k * k * (J0 - J1 / z);
    } else {
        const double kap = sqrt(-q);
        const double z = kap * r;
        double K0, K1;
        bessel_k01(z, &K0, &K1);
        const double inv2pi = 0.5 / kPi;
        out[0] = -K0 * inv2pi;
        out[1] = 0.0;
        out[2] = kap * K1 * inv2pi;
        out[3] = 0.0;
        out[4] = -kap * kap * (K0 + K1 / z) * inv2pi;
        out[5] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// Complex q (complex c): K0(w), K1(w) for complex w, -pi < arg w < pi, and the
// kernels through them.  With k = sqrt(q) on the branch arg q in (-pi/2, 3pi/2]
// (arg k in (-pi/4, 3pi/4]) and kc = -i k, the Helmholtz kernel is
//   g = -(i/4) H0(k r) = -K0(kc r)/(2 pi),  g' = kc K1(kc r)/(2 pi),
//   g'' = -kc^2 (K0(kc r) + K1(kc r)/(kc r))/(2 pi)          (H_nu(z) = (2/pi) i^(-nu-1) K_nu(-i z)),
// the real q < 0 formulas with kappa -> kc; w = kc r has arg w in (-3pi/4, pi/4].
//   |w| <= 2: the ascending series of bessel_k01 in complex arithmetic (principal log;
//     the cut, on the negative real axis of w, is outside that sector);
//   |w| > 2: K_nu(w) = int_0^inf exp(-w cosh t) cosh(nu t) dt along the contour
//     t: 0 -> -i beta -> -i beta + inf (exp(-w cosh t) is entire, so the contour
//     continues K analytically to Re w <= 0).  The horizontal ray decays like
//     exp(-|w| e^s cos(theta - beta)/2) and oscillates like exp(-i |w| e^s sin(theta - beta)/2),
//     theta = arg w.  The vertical piece to -i beta passes values up to
//     e^{|w| cos theta (1 - cos beta)} |K|: beta = theta where Re w <= 0 (no excess), else
//     the largest |beta| <= |theta| with that factor at most e^2, which keeps the ray's
//     oscillation slow against its decay without cancellation.  Gauss-Legendre:
//     ceil(|beta| |w| / 8) 16-point panels on the vertical piece, 4 on the ray [0, S],
//     S = ln(2 (40 + |w|)/(|w| cos(theta - beta))) + 1/2.  Measured against scipy over
//     2 < |w| < 40 in the sector (and along arg w = -pi/2): 1.4e-14 relative.
// g16t, g16w: the 16-point Gauss-Legendre nodes and weights on [-1, 1].
struct cplx_d {
    double re, im;
};
__host__ __device__ inline cplx_d cz_mul(cplx_d a, cplx_d b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ inline cplx_d cz_add(cplx_d a, cplx_d b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ inline cplx_d cz_sub(cplx_d a, cplx_d b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ inline cplx_d cz_scale(cplx_d a, double s) { return {a.re * s, a.im * s}; }
__host__ __device__ inline cplx_d cz_exp(cplx_d a) {
    const double m = exp(a.re);
    return {m * cos(a.im), m * sin(a.im)};
}
__host__ __device__ inline cplx_d cz_rcp(cplx_d a) {
    const double d = 1.0 / (a.re * a.re + a.im * a.im);
    return {a.re * d, -a.im * d};
}

__host__ __device__ inline void bessel_k01_c(cplx_d w, const double* g16t, const double* g16w,
                                             cplx_d* k0v, cplx_d* k1v)
{
    const double u = sqrt(w.re * w.re + w.im * w.im);
    if (u <= 2.0) {
        constexpr SeriesK01d C = series_k01_d();
        const cplx_d t = cz_scale(cz_mul(w, w), 0.25);
        cplx_d i0 = {C.c0[kSeriesK01d - 1], 0.0}, s0 = {C.d0[kSeriesK01d - 1], 0.0};
        cplx_d i1s = {C.c1[kSeriesK01d - 1], 0.0}, s1 = {C.d1[kSeriesK01d - 1], 0.0};
        for (int j = kSeriesK01d - 2; j >= 0; --j) {
            i0 = cz_add(cz_mul(i0, t), cplx_d{C.c0[j], 0.0});
            s0 = cz_add(cz_mul(s0, t), cplx_d{C.d0[j], 0.0});
            i1s = cz_add(cz_mul(i1s, t), cplx_d{C.c1[j], 0.0});
            s1 = cz_add(cz_mul(s1, t), cplx_d{C.d1[j], 0.0});
        }
        const cplx_d lg = {log(0.5 * u), atan2(w.im, w.re)};        // log(w/2)
        *k0v = cz_sub(s0, cz_mul(lg, i0));
        const cplx_d hw = cz_scale(w, 0.5);
        *k1v = cz_sub(cz_add(cz_rcp(w), cz_mul(lg, cz_mul(hw, i1s))), cz_mul(cz_scale(w, 0.25), s1));
        return;
    }
    const double th = atan2(w.im, w.re);
    // the largest shift |beta| <= |theta| whose vertical piece stays within e^2 of |K|
    // (u cos theta (1 - cos beta) <= 2); all of theta where Re w <= 0
    double beta = th;
    if (cos(th) > 0.0) {
        const double lim = fmax(-1.0, fmin(1.0, 1.0 - 2.0 / (u * cos(th))));
        beta = copysign(fmin(fabs(th), acos(lim)), th);
    }
    cplx_d a0 = {0.0, 0.0}, a1 = {0.0, 0.0};
    // vertical piece: t = -i tau, tau from 0 to beta, dt = -i dtau, cosh t = cos tau
    const int nv = beta != 0.0 ? (int)fmin(64.0, fmax(1.0, ceil(fabs(beta) * u / 8.0))) : 0;
    cplx_d v0 = {0.0, 0.0}, v1 = {0.0, 0.0};
    for (int p = 0; p < nv; ++p) {
        const double lo = beta * p / nv, hi = beta * (p + 1) / nv, h = 0.5 * (hi - lo);
        for (int q = 0; q < 16; ++q) {
            const double tau = lo + h * (g16t[q] + 1.0), ct = cos(tau);
            const cplx_d e = cz_scale(cz_exp(cz_scale(w, -ct)), h * g16w[q]);
            v0 = cz_add(v0, e);
            v1 = cz_add(v1, cz_scale(e, ct));
        }
    }
    a0 = {v0.im, -v0.re};                                    // times -i
    a1 = {v1.im, -v1.re};
    // the ray t = s - i beta, s in [0, S]: cosh t = cosh s cos beta - i sinh s sin beta
    const double S = log(2.0 * (40.0 + u) / (u * cos(th - beta))) + 0.5;
    const double cb = cos(beta), sb = sin(beta);
    for (int p = 0; p < 4; ++p) {
        const double lo = S * p / 4, h = 0.125 * S;
        for (int q = 0; q < 16; ++q) {
            const double sv = lo + h * (g16t[q] + 1.0);
            const cplx_d ch = {cosh(sv) * cb, -sinh(sv) * sb};
            const cplx_d e = cz_scale(cz_exp(cz_scale(cz_mul(w, ch), -1.0)), h * g16w[q]);
            a0 = cz_add(a0, e);
            a1 = cz_add(a1, cz_mul(e, ch));
        }
    }
    *k0v = a0;
    *k1v = a1;
}

// (g, g', g'') as (re, im) pairs for complex q (q.im != 0; see above).
__host__ __device__ inline void green_scaled_cz(double r, cplx_d q, const double* g16t,
                                                const double* g16w, double* out)
{
    // principal root without cancellation (the larger part from |q| + |Re q|, the other
    // as Im q / (2 that part)), then the branch arg q in (-pi/2, 3pi/2]: negate where
    // arg q < -pi/2
    const double mod = sqrt(q.re * q.re + q.im * q.im);
    double kr, ki;
    if (q.re >= 0.0) {
        kr = sqrt(0.5 * (mod + q.re));
        ki = q.im / (2.0 * kr);
    } else {
        ki = copysign(sqrt(0.5 * (mod - q.re)), q.im);
        kr = q.im / (2.0 * ki);
    }
    if (q.im < 0.0 && q.re <= 0.0) { kr = -kr; ki = -ki; }
    const cplx_d kc = {ki, -kr};                             // -i k
    const cplx_d w = cz_scale(kc, r);
    cplx_d K0, K1;
    bessel_k01_c(w, g16t, g16w, &K0, &K1);
    const double inv2pi = 0.5 / kPi;
    const cplx_d g = cz_scale(K0, -inv2pi);
    const cplx_d g1 = cz_scale(cz_mul(kc, K1), inv2pi);
    const cplx_d g2 = cz_scale(cz_mul(cz_mul(kc, kc), cz_add(K0, cz_mul(K1, cz_rcp(w)))), -inv2pi);
    out[0] = g.re; out[1] = g.im;
    out[2] = g1.re; out[3] = g1.im;
    out[4] = g2.re; out[5] = g2.im;
}

// green_scaled for any real q: q = 0 is the c~ = 0 Green's function log(r)/(2 pi)
// (g' = 1/(2 pi r), g'' = -1/(2 pi r^2)).  A coefficient c whose sign changes
// over the surface passes through q = 0, where the Helmholtz kernel has no limit
// (it grows like log |q|, Sec. 4.2); the paper's G for c~ = 0 is taken there.
__host__ __device__ inline void green_scaled_any(double r, double q, double* out)
{
    if (q != 0.0) {
        green_scaled(r, q, out);
        return;
    }
    const double inv2pi = 0.5 / kPi;
    out[0] = log(r) * inv2pi;
    out[2] = inv2pi / r;
    out[4] = -inv2pi / (r * r);
    out[1] = out[3] = out[5] = 0.0;
}

// One source's a(y) R and a(y) K for real q(y) = c(y)/a(y), as (re, im) pairs
// out[0..1] = a(y) R, out[2..3] = a(y) K (eq. explicit_remainder with
// a(y) G = g(r; k(y)), k(y)^2 = q(y)), r = x - y:
//   a(y) R = (gb . r^) g' - a(x) (g'' - g'/r) (n.r^)^2 - 2 a(x) H(x) (n.r^) g'
//            + (c(x) - a(x) q(y)) g,          a(y) K = g,
// gb = grad_G a(x), n and H the target's normal and mean curvature.
__host__ __device__ inline void pair_rk_c(double rx, double ry, double rz, double nx, double ny,
                                          double nz, double H, double a, double gbx, double gby,
                                          double gbz, double c, double q, double* out)
{
    const double r = sqrt(rx * rx + ry * ry + rz * rz);
    const double inv_r = 1.0 / r;
    double g[6];
    green_scaled_any(r, q, g);
    const double nr = (nx * rx + ny * ry + nz * rz) * inv_r;
    const double gr = (gbx * rx + gby * ry + gbz * rz) * inv_r;
    const double t2 = a * nr * nr;
    const double t1 = gr - 2.0 * a * H * nr;
    const double t0 = c - a * q;
    out[0] = t1 * g[2] - t2 * (g[4] - g[2] * inv_r) + t0 * g[0];
    out[1] = t1 * g[3] - t2 * (g[5] - g[3] * inv_r) + t0 * g[1];
    out[2] = g[0];
    out[3] = g[1];
}

// pair_rk_c with complex c(x) and q(y) (out as in pair_rk_c): the real-q path when
// q is real, the complex kernels otherwise.
__host__ __device__ inline void pair_rk_cz(double rx, double ry, double rz, double nx, double ny,
                                           double nz, double H, double a, double gbx, double gby,
                                           double gbz, cplx_d c, cplx_d q, const double* g16t,
                                           const double* g16w, double* out)
{
    const double r = sqrt(rx * rx + ry * ry + rz * rz);
    const double inv_r = 1.0 / r;
    double g[6];
    if (q.im == 0.0) green_scaled_any(r, q.re, g);
    else green_scaled_cz(r, q, g16t, g16w, g);
    const double nr = (nx * rx + ny * ry + nz * rz) * inv_r;
    const double gr = (gbx * rx + gby * ry + gbz * rz) * inv_r;
    const double t2 = a * nr * nr;
    const double t1 = gr - 2.0 * a * H * nr;
    const cplx_d t0 = {c.re - a * q.re, c.im - a * q.im};       // c(x) - a(x) q(y)
    out[0] = t1 * g[2] - t2 * (g[4] - g[2] * inv_r) + (t0.re * g[0] - t0.im * g[1]);
    out[1] = t1 * g[3] - t2 * (g[5] - g[3] * inv_r) + (t0.re * g[1] + t0.im * g[0]);
    out[2] = g[0];
    out[3] = g[1];
}

// ---------------------------------------------------------------------------
// float32 versions for the per-pair smooth sums.  Same methods, tuned to
// float32: the series for x < 2 with ten unrolled terms (t = x^2/4 <= 1, so
// the tail is below 1/(10!)^2) and constant-folded coefficients; the trapezoid
// rule for x >= 2 with h = min(1/2, pi^2/(18.5 + x)) (error O(exp(x - pi^2/h))
// below 1e-8 relative), cut where the integrand falls below e^-18.5, at most
// 7 terms; sinh(j h/2), cosh(j h/2) by the addition formulas.  K0 and K1
// underflow float32 beyond x = 87 and return 0.  Measured against the exact
// functions at the float32 argument: <= 7e-7 relative.
// ---------------------------------------------------------------------------

// Coefficients of the float32 series, computed at compile time:
// f0[j] = 1/(j+1)^2, f1[j] = 1/((j+1)(j+2)) (ratios of consecutive terms),
// p0[j] = psi(j+1), p1[j] = psi(j+1) + psi(j+2).
struct SeriesK01 {
    float f0[10], f1[10], p0[10], p1[10];
};

__host__ __device__ constexpr SeriesK01 series_k01()
{
    SeriesK01 c{};
    double harm = 0.0;
    for (int j = 0; j < 10; ++j) {
        const double psi1 = -kEulerGamma + harm;
        c.p0[j] = (float)psi1;
        c.p1[j] = (float)(2.0 * psi1 + 1.0 / (j + 1));
        c.f0[j] = (float)(1.0 / ((j + 1.0) * (j + 1.0)));
        c.f1[j] = (float)(1.0 / ((j + 1.0) * (j + 2.0)));
        harm += 1.0 / (j + 1);
    }
    return c;
}

__host__ __device__ inline void bessel_k01_f32(float x, float* k0v, float* k1v)
{
    if (x < 2.0f) {
        constexpr SeriesK01 C = series_k01();
        const float t = 0.25f * x * x;
        float a0 = 1.0f, a1 = 1.0f, i0 = 0.0f, i1s = 0.0f, s0 = 0.0f, s1 = 0.0f;
#pragma unroll
        for (int j = 0; j < 10; ++j) {
            i0 += a0;
            i1s += a1;
            s0 = fmaf(C.p0[j], a0, s0);
            s1 = fmaf(C.p1[j], a1, s1);
            a0 *= t * C.f0[j];
            a1 *= t * C.f1[j];
        }
        const float lg = logf(0.5f * x);
        *k0v = fmaf(-lg, i0, s0);
        *k1v = 1.0f / x + lg * (0.5f * x * i1s) - 0.25f * x * s1;
        return;
    }
    if (!(x <= 87.0f)) {                // underflow, or NaN passed through
        *k0v = *k1v = (x > 87.0f) ? 0.0f : x;
        return;
    }
    const float h = fminf(0.5f, (float)(kPi * kPi) / (18.5f + x));
    const int n = (int)fminf(16.0f, ceilf(acoshf(1.0f + 18.5f / x) / h));   // <= 7 here
    const float sh1 = sinhf(0.5f * h), ch1 = coshf(0.5f * h);
    float sh = 0.0f, ch = 1.0f, S0 = 0.5f, S1 = 0.5f;
    for (int j = 1; j <= n; ++j) {
        const float shn = fmaf(sh, ch1, ch * sh1);
        ch = fmaf(ch, ch1, sh * sh1);
        sh = shn;
        const float s2 = sh * sh;
        const float e = expf(-2.0f * x * s2);
        S0 += e;
        S1 = fmaf(e, fmaf(2.0f, s2, 1.0f), S1);
    }
    const float ex = expf(-x);
    *k0v = h * S0 * ex;
    *k1v = h * S1 * ex;
}

// float32 (g, g', g'') as in green_scaled, for q = c~/a~ real and non-zero.
__host__ __device__ inline void green_scaled_f32(float r, float q, float* out)
{
    if (q > 0.0f) {
        const float k = sqrtf(q);
        const float z = k * r;
        const float J0 = j0f(z), Y0 = y0f(z), J1 = j1f(z), Y1 = y1f(z);
        const float kk = 0.25f * k * k;
        out[0] = 0.25f * Y0;
        out[1] = -0.25f * J0;
        out[2] = -0.25f * k * Y1;
        out[3] = 0.25f * k * J1;
        out[4] = -kk * (Y0 - Y1 / z);
        out[5] = kk * (J0 - J1 / z);
    } else {
        const float kap = sqrtf(-q);
        const float z = kap * r;
        float K0, K1;
        bessel_k01_f32(z, &K0, &K1);
        const float inv2pi = (float)(0.5 / kPi);
        out[0] = -K0 * inv2pi;
        out[1] = 0.0f;
        out[2] = kap * K1 * inv2pi;
        out[3] = 0.0f;
        out[4] = -kap * kap * (K0 + K1 / z) * inv2pi;
        out[5] = 0.0f;
    }
}

// One source's float32 contribution to the smooth sums of R and K for real c != 0
// (eq. explicit_remainder with a(y) G = g(r; k_y), k_y^2 = q = c(y)/a(y)):
//   a(y) R = gb . r^ g' - a(x) (g'' - g'/r) (n.r)^2/r^2 - 2 a(x) H(x) (n.r^) g'
//            + (c(x) - a(x) q) g,        a(y) K = g,
// gb = grad_G a(x) (+ b(x) for advection).  The source weight s = w sigma / a(y)
// is complex; acc[0..3] += Re, Im of a(y) R s and of a(y) K s.
__host__ __device__ inline void pair_rk_c_f32(float rx, float ry, float rz, float nx, float ny,
                                              float nz, float H, float a, float gbx, float gby,
                                              float gbz, float c, float q, float s_re, float s_im,
                                              float* acc)
{
    const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
    const float r = sqrtf(r2);
    const float inv_r = 1.0f / r;
    float g[6];
    green_scaled_f32(r, q, g);
    const float nr = fmaf(nx, rx, fmaf(ny, ry, nz * rz)) * inv_r;       // n . r^
    const float gr = fmaf(gbx, rx, fmaf(gby, ry, gbz * rz)) * inv_r;    // gb . r^
    const float t2 = a * nr * nr;                                        // a (n.r)^2 / r^2
    const float t1 = fmaf(-2.0f * a * H, nr, gr);                        // gb.r^ - 2 a H n.r^
    const float t0 = fmaf(-a, q, c);                                     // c(x) - a(x) q
    // a(y) R = t1 g' - t2 (g'' - g'/r) + t0 g, componentwise in (re, im)
    const float R_re = fmaf(t1, g[2], fmaf(-t2, fmaf(-g[2], inv_r, g[4]), t0 * g[0]));
    const float R_im = fmaf(t1, g[3], fmaf(-t2, fmaf(-g[3], inv_r, g[5]), t0 * g[1]));
    acc[0] += R_re * s_re - R_im * s_im;
    acc[1] += R_re * s_im + R_im * s_re;
    acc[2] += g[0] * s_re - g[1] * s_im;
    acc[3] += g[0] * s_im + g[1] * s_re;
}

}  // namespace pm_green
