// Float-float (FP32-pair) arithmetic shared by the float-float smooth sums.
//
// A value is the unevaluated sum h + l of two floats (about 48 significant
// bits).  The building blocks are the error-free transformations TwoSum
// (Knuth), Fast2Sum (Dekker, |a| >= |b| or a = 0) and TwoProduct through FMA.
//
// Most operations here are "lazy": the result is left unnormalised, its low
// word possibly larger than half an ulp of the high word.  Products and sums
// of such pairs keep float-float accuracy while the low word stays small in
// absolute terms next to what the result needs; every sum that can cancel
// (dot products, the bracket of the remainder term) is renormalised with
// ff_norm before it is multiplied.
//
// Coordinates of the parametrix sums use a split of their own (pm_ff_grid;
// the remainder sums keep plain pairs, see pm_ffsum.cu): the high word is
// x rounded to the grid 2^(E - 22), 2^E >= max |x|, and the low word is the
// float nearest x - hi.  Two high words then differ by an exact float, so a
// coordinate difference needs no TwoSum: ff_grid_sub.
#pragma once

#include <cuda_runtime.h>

namespace pmff {

struct ff {
    float h, l;
};

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// requires |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ ff ff_norm(ff a) {
    ff r;
    fast_two_sum(a.h, a.l, r.h, r.l);
    return r;
}

__device__ __forceinline__ ff ff_mul_lazy(ff a, ff b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return ff{p, e};
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) { return ff_norm(ff_mul_lazy(a, b)); }

// (h + l)^2 = h^2 + l (2h + l): the l^2 term is kept, so the square stays
// accurate when l is as large as h (coordinate differences of nearby points)
__device__ __forceinline__ ff ff_sqr_lazy(ff a) {
    const float p = a.h * a.h;
    float e = fmaf(a.h, a.h, -p);
    e = fmaf(a.l, fmaf(2.f, a.h, a.l), e);
    return ff{p, e};
}

__device__ __forceinline__ ff ff_add_lazy(ff a, ff b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    return ff{s, e + (a.l + b.l)};
}

// a + b when |a.h| >= |b.h| or a.h = 0
__device__ __forceinline__ ff ff_add_ordered_lazy(ff a, ff b) {
    float s, e;
    fast_two_sum(a.h, b.h, s, e);
    return ff{s, e + (a.l + b.l)};
}

// 1/a: y = rcp(a.h) and one Newton step y + y (1 - a y), the residual 1 - a y
// formed with the exact product a.h y = p + ep; returned unnormalised as (y, y res)
__device__ __forceinline__ ff ff_rcp_lazy(ff a) {
    const float y = rcp_approx(a.h);
    const float p = a.h * y;
    const float ep = fmaf(a.h, y, -p);
    const float res = ((1.f - p) - ep) - a.l * y;
    return ff{y, y * res};
}

constexpr int kLogTable = 128;

// ln(x) for x = h + l > 0 with x.h a normal float, after Tang ("Table-driven
// implementation of the logarithm function in IEEE floating-point arithmetic",
// ACM TOMS 16, 1990): x = 2^e m, m in [1, 2); m = c_k (1 + t), c_k = 1 + (k +
// 1/2)/128 from the top seven fraction bits, |t| <= 2^-8; ln x = e ln 2 +
// ln c_k + ln(1 + t), ln(1 + t) = t - t^2/2 + t^3 (1/3 - t/4 + t^2/5 - t^3/6)
// (truncation below 2^-56).  tab[k] = (1/c_k hi, lo, ln c_k hi, lo).
// e, m and k are read from the bits of x.h.  Sums whose order of magnitude is
// known use Fast2Sum: |e ln 2| >= ln 2 > ln c_k unless e = 0, and
// |t^2/2 - t^3/3 ...| <= 2^-9 |t|.  The result is unnormalised.
__device__ __forceinline__ ff ff_log_lazy(ff x, const float4* __restrict__ tab) {
    const unsigned bits = __float_as_uint(x.h);
    const int ebias = (int)(bits >> 23);                      // biased exponent (x.h > 0)
    const float mh = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);
    const float sc = __uint_as_float((unsigned)(254 - ebias) << 23);   // 2^-e
    const ff m{mh, x.l * sc};
    const float4 T = tab[(bits >> 16) & 0x7Fu];
    const ff p = ff_mul_lazy(m, ff{T.x, T.y});                // m / c_k = 1 + t
    const ff t{p.h - 1.f, p.l};                               // p.h - 1 is exact (Sterbenz)
    const ff t2 = ff_sqr_lazy(t);
    const float tf = t.h + t.l;                               // t to float accuracy (t.l can be
                                                              // a sizeable part of t.h here)
    const float poly = fmaf(fmaf(fmaf(-1.f / 6.f, tf, 0.2f), tf, -0.25f), tf, 1.f / 3.f);
    const float cubic = tf * tf * tf * poly;
    const ff small{-0.5f * t2.h, fmaf(-0.5f, t2.l, cubic)};
    // e ln 2 = L2H e + L2L e; the FMA recovers the rounding of L2H e exactly
    const float L2H = 0.693147182464599609375f;
    const float L2L = -1.904654323148236e-09f;
    const float ef = (float)(ebias - 127);
    const float eh = L2H * ef;
    const ff el{eh, fmaf(L2L, ef, fmaf(L2H, ef, -eh))};
    return ff_add_lazy(ff_add_ordered_lazy(el, ff{T.z, T.w}), ff_add_ordered_lazy(t, small));
}

__device__ __forceinline__ ff ff_from_double(double v) {
    const float h = (float)v;
    return ff{h, (float)(v - (double)h)};
}

// a - b for plain float-float values, normalised: where the high words cancel
// the low word is then no larger than half an ulp of the result
__device__ __forceinline__ ff ff_sub(ff a, ff b) {
    float s, e;
    two_sum(a.h, -b.h, s, e);
    return ff_norm(ff{s, e + (a.l - b.l)});
}

// X - Y for grid-split coordinates, Y = (yh, yl): the high words differ by an
// exact float, so Fast2Sum (|X.h - yh| is 0 or at least the grid, |X.l - yl|
// at most the grid) renormalises the pair; products with it then keep
// float-float accuracy.  Absolute error about 2^(E - 46).
__device__ __forceinline__ ff ff_grid_sub(ff X, float yh, float yl) {
    ff r;
    fast_two_sum(X.h - yh, X.l - yl, r.h, r.l);
    return r;
}

// Coordinate split on the grid g (a power of two, see the file header).
__device__ __forceinline__ ff ff_grid_split(double v, double g) {
    const double hi = rint(v / g) * g;
    return ff{(float)hi, (float)(v - hi)};
}

}  // namespace pmff
