// Double-double arithmetic on the FP64 pipe: a value is the unevaluated sum h + l of
// two doubles with |l| <= ulp(h)/2, about 106 significant bits.  Written from the
// error-free transformations of Dekker (1971) and Knuth (TwoSum), with the
// normalisation and the accurate addition of Hida, Li and Bailey's double-double
// scheme (2001); exp, log, sin and cos by argument reduction, Taylor series and a
// Newton step, as described there.  Used by the device build of the VDIM
// correction, whose entries are small differences of large numbers.
#pragma once

struct DD {
    double h, l;
};

#include "dd_consts.h"

__device__ __forceinline__ DD dd(double a) { return DD{a, 0.0}; }

__device__ __forceinline__ DD quick_two_sum(double a, double b) {       // |a| >= |b|
    const double s = a + b;
    return DD{s, b - (s - a)};
}

__device__ __forceinline__ DD two_sum(double a, double b) {
    const double s = a + b;
    const double bb = s - a;
    return DD{s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ DD two_prod(double a, double b) {
    const double p = a * b;
    return DD{p, fma(a, b, -p)};
}

__device__ __forceinline__ DD dd_add(DD a, DD b) {
    DD s = two_sum(a.h, b.h);
    DD t = two_sum(a.l, b.l);
    s.l += t.h;
    s = quick_two_sum(s.h, s.l);
    s.l += t.l;
    return quick_two_sum(s.h, s.l);
}

__device__ __forceinline__ DD dd_neg(DD a) { return DD{-a.h, -a.l}; }
__device__ __forceinline__ DD dd_sub(DD a, DD b) { return dd_add(a, dd_neg(b)); }

__device__ __forceinline__ DD dd_add_d(DD a, double b) {
    DD s = two_sum(a.h, b);
    s.l += a.l;
    return quick_two_sum(s.h, s.l);
}

__device__ __forceinline__ DD dd_mul(DD a, DD b) {
    DD p = two_prod(a.h, b.h);
    p.l += a.h * b.l + a.l * b.h;
    return quick_two_sum(p.h, p.l);
}

__device__ __forceinline__ DD dd_mul_d(DD a, double b) {
    DD p = two_prod(a.h, b);
    p.l += a.l * b;
    return quick_two_sum(p.h, p.l);
}

// exact scaling by a power of two
__device__ __forceinline__ DD dd_ldexp(DD a, int e) { return DD{ldexp(a.h, e), ldexp(a.l, e)}; }

__device__ __forceinline__ DD dd_div(DD a, DD b) {
    const double q1 = a.h / b.h;
    DD r = dd_sub(a, dd_mul_d(b, q1));
    const double q2 = r.h / b.h;
    r = dd_sub(r, dd_mul_d(b, q2));
    const double q3 = r.h / b.h;
    DD q = quick_two_sum(q1, q2);
    return dd_add_d(q, q3);
}

__device__ __forceinline__ DD dd_sqrt(DD a) {                           // a > 0
    const double x = sqrt(a.h);
    // one Newton step from the double root: x + (a - x^2) / (2 x)
    const DD x2 = two_prod(x, x);
    const DD r = dd_sub(a, x2);
    return dd_add_d(DD{x, 0.0}, r.h / (2.0 * x));
}

// e^a - 1 for |a| small (Taylor series to 1/12!)
__device__ __forceinline__ DD dd_expm1_small(DD r) {
    DD s = r, t = r;
#pragma unroll 1
    for (int n = 2; n <= 12; ++n) {
        t = dd_mul(t, r);
        s = dd_add(s, dd_mul(t, dd_inv_fact[n]));
    }
    return s;
}

// e^a = 2^k e^r, a = k ln 2 + r, e^r from (r / 2^10) by ten squarings of 1 + s
__device__ DD dd_exp(DD a) {
    const DD ln2 = DD_LN2;
    const double k = rint(a.h / ln2.h);
    DD r = dd_sub(a, dd_mul_d(ln2, k));
    r = dd_ldexp(r, -10);
    DD s = dd_expm1_small(r);
#pragma unroll 1
    for (int i = 0; i < 10; ++i) s = dd_add(dd_ldexp(s, 1), dd_mul(s, s));   // e^{2x} - 1 = 2 s + s^2
    return dd_ldexp(dd_add_d(s, 1.0), (int)k);
}

// log a (a > 0): y = log(a_h) in double, then one Newton step y + a e^{-y} - 1
__device__ DD dd_log(DD a) {
    const double y = log(a.h);
    const DD e = dd_exp(DD{-y, 0.0});
    return dd_add_d(dd_add_d(dd_mul(a, e), -1.0), y);
}

// sin and cos of a (|a| up to a few hundred): a = q pi/2 + r, |r| <= pi/4, Taylor series
__device__ void dd_sincos(DD a, DD& s, DD& c) {
    const DD pi2 = DD_PI_2;
    const double q = rint(a.h / pi2.h);
    const DD r = dd_sub(a, dd_mul_d(pi2, q));
    const DD r2 = dd_mul(r, r);
    DD p = dd(1.0);                             // r^n, n even
    DD ss = r, cc = dd(1.0);
#pragma unroll 1
    for (int n = 2; n <= 28; n += 2) {
        p = dd_mul(p, r2);
        const DD tc = dd_mul(p, dd_inv_fact[n]);
        const DD ts = dd_mul(dd_mul(p, r), dd_inv_fact[n + 1]);
        if ((n >> 1) & 1) { cc = dd_sub(cc, tc); ss = dd_sub(ss, ts); }
        else { cc = dd_add(cc, tc); ss = dd_add(ss, ts); }
    }
    const int m = ((int)q) & 3;
    if (m == 0) { s = ss; c = cc; }
    else if (m == 1) { s = cc; c = dd_neg(ss); }
    else if (m == 2) { s = dd_neg(ss); c = dd_neg(cc); }
    else { s = dd_neg(cc); c = ss; }
}

struct CDD {
    DD re, im;
};

__device__ __forceinline__ CDD cdd_mul(CDD a, CDD b) {
    return CDD{dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im)), dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
}
__device__ __forceinline__ CDD cdd_scale(CDD a, DD s) { return CDD{dd_mul(a.re, s), dd_mul(a.im, s)}; }
