// Double-single ("float-float") arithmetic for the complex128 fused pass.
//
// The paper keeps the register in double precision (Sec. 2.1).  On this GPU
// the double-precision pipe issues about one sixty-fourth of the
// single-precision rate, and a fused pass of the random-circuit workload
// does 16 double flops per amplitude per gate, so the complex128 pass is
// bound by that pipe.  The complex128 state therefore stays in double
// precision in memory (the paper's layout: 16-byte (re, im) amplitudes), and
// a pass converts each amplitude at its load into a pair of floats whose sum
// carries 48 significant bits, applies the gates with single-precision
// instructions and error-free transformations, and converts back to double
// at the store:
//
//   * TwoProd (exact product, from the fused multiply-add): a*b = p + e with
//     p = fl(a*b), e = fma(a, b, -p);
//   * TwoSum (Knuth, branch-free): a + b = s + e exactly;
//   * FastTwoSum (Dekker, |a| >= |b|): a + b = s + e exactly.
//
// A real output of a 2x2 update is a four-term dot product: the products of
// the high parts are exact pairs (p_k, e_k), the high parts p_k are summed
// with TwoSum, and every low-order term (the e_k, the cross terms a.h*b.l and
// a.l*b.h, and the TwoSum errors) is summed in single precision; FastTwoSum
// renormalises the result.  Its error is a few units of 2^-48 of the largest
// term, against 2^-53 for double precision.
//
// The conversions use integer instructions only (no double-precision
// instruction runs in the pass).  Every function here is written for both
// the host and the device, so the host tests check the conversions and the
// arithmetic bit for bit against exact rational arithmetic.
#pragma once

#include <stdint.h>
#include <string.h>

#ifndef __CUDACC__
#include <cmath>
#define QS_HD inline
#else
#define QS_HD __host__ __device__ __forceinline__
#endif

namespace qs {
namespace ds {

// Operations with one rounding each, never contracted into an FMA.
#if defined(__CUDA_ARCH__)
QS_HD float add(float a, float b) { return __fadd_rn(a, b); }
QS_HD float sub(float a, float b) { return __fsub_rn(a, b); }
QS_HD float mul(float a, float b) { return __fmul_rn(a, b); }
QS_HD float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
QS_HD uint32_t fbits(float f) { return __float_as_uint(f); }
QS_HD float bitsf(uint32_t u) { return __uint_as_float(u); }
QS_HD uint64_t dbits(double d) { return uint64_t(__double_as_longlong(d)); }
QS_HD double bitsd(uint64_t u) { return __longlong_as_double((long long)u); }
QS_HD float u2f(uint32_t u) { return __uint2float_rn(u); }
QS_HD int f2i(float f) { return __float2int_rn(f); }
#else
// Host builds of these helpers must be compiled without floating-point
// contraction (-ffp-contract=off) so that each line rounds once.
QS_HD float add(float a, float b) { volatile float r = a + b; return r; }
QS_HD float sub(float a, float b) { volatile float r = a - b; return r; }
QS_HD float mul(float a, float b) { volatile float r = a * b; return r; }
QS_HD float fma(float a, float b, float c) { return std::fmaf(a, b, c); }
QS_HD uint32_t fbits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
QS_HD float bitsf(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
QS_HD uint64_t dbits(double d) { uint64_t u; memcpy(&u, &d, 8); return u; }
QS_HD double bitsd(uint64_t u) { double d; memcpy(&d, &u, 8); return d; }
QS_HD float u2f(uint32_t u) { return float(u); }   // exact for u < 2^24, else round to nearest even
QS_HD int f2i(float f) { return int(std::nearbyintf(f)); }
#endif

// a + b = s + e exactly (Knuth's TwoSum, no condition on the operands).
QS_HD void two_sum(float a, float b, float &s, float &e) {
    s = add(a, b);
    const float bb = sub(s, a);
    e = add(sub(a, sub(s, bb)), sub(b, bb));
}

// a + b = s + e exactly when |a| >= |b| or a == 0 (Dekker's FastTwoSum).
QS_HD void fast_two_sum(float a, float b, float &s, float &e) {
    s = add(a, b);
    e = sub(b, sub(s, a));
}

// Double -> (h, l), h + l equal to d truncated to 48 significant bits.
// h is d truncated to a float's 24 bits (same sign as d); l is the next 24
// bits of d (rounded to nearest from the remaining 29 bits), of the same
// sign.  Exponent ranges: |d| >= 2^-126 gives h exactly; |d| < 2^-126 gives
// h = l = 0 (an absolute error below 2^-126); |d| < 2^-74 drops l (an
// absolute error below 2^-97).  |d| must be below 2^127 (amplitudes of a
// state are at most 1 in magnitude).
QS_HD void split(double d, float &h, float &l) {
    const uint64_t b = dbits(d);
    const uint32_t hi = uint32_t(b >> 32), lo = uint32_t(b);
    const uint32_t e = (hi >> 20) & 0x7ffu;
    const uint32_t sgn = hi & 0x80000000u;
    // exponent field rebased from 1023 to 127 modulo 2^9, top 23 mantissa bits
    const uint32_t hb = (((hi << 3) | (lo >> 29)) - 0xC0000000u) | sgn;
    h = e > 896u ? bitsf(hb) : 0.0f;
    // the remaining 29 mantissa bits times 2^(e - 1075)
    const float r = u2f(lo & 0x1fffffffu);
    const float sc = bitsf((e - 948u) << 23);
    const float lm = mul(r, sc);
    l = e > 948u ? bitsf(fbits(lm) | sgn) : 0.0f;
}

// (h, l) -> the double nearest h + l, for a pair with |l| <= ulp(h) (what
// every arithmetic function here returns).  |h| < 2^-126 gives 0; |h| <
// 2^-75 gives h alone (an absolute error below 2^-99).
QS_HD double join(float h, float l) {
    const uint32_t hb = fbits(h);
    const uint32_t ef = (hb >> 23) & 0xffu;
    const uint32_t sgn = hb & 0x80000000u;
    // h in double: exponent 127 -> 1023, mantissa shifted into place
    uint32_t dhi = (((hb & 0x7fffffffu) >> 3) + 0x38000000u);
    uint32_t dlo = hb << 29;
    // l in units of h's double ulp 2^(ef - 127 - 52): l * 2^(179 - ef)
    const float sc = bitsf((306u - ef) << 23);
    int k = f2i(mul(l, sc));
    if (sgn) k = -k;                                   // k now adds to the magnitude
    if ((hb & 0x7fffffu) == 0u && k < 0) k *= 2;       // below a power of two the ulp halves
    const uint64_t mag = ((uint64_t(dhi) << 32) | dlo) + uint64_t(int64_t(k));
    const double r = bitsd(mag | (uint64_t(sgn) << 32));
    if (ef == 0u) return 0.0;
    if (ef < 52u) return bitsd((uint64_t(dhi | sgn) << 32) | dlo);
    return r;
}

// Sum over k < 4 of a_k * b_k (a_k = (ah[k], al[k]), b_k likewise), the
// result renormalised: |l| <= ulp(h) / 2.  The product of the low parts is
// dropped (2^-48 of its term).
QS_HD void dot4(const float (&ah)[4], const float (&al)[4], const float (&bh)[4], const float (&bl)[4], float &h,
                float &l) {
#ifndef QS_DS_CHAIN
    // pairwise: the high products summed as (p0 + p1) + (p2 + p3), the
    // low-order terms in two independent chains, for instruction-level
    // parallelism
    float p[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) p[k] = mul(ah[k], bh[k]);
    float la = fma(ah[0], bh[0], -p[0]), lb = fma(ah[2], bh[2], -p[2]);
    la = fma(ah[0], bl[0], la);
    lb = fma(ah[2], bl[2], lb);
    la = fma(al[0], bh[0], la);
    lb = fma(al[2], bh[2], lb);
    la = add(la, fma(ah[1], bh[1], -p[1]));
    lb = add(lb, fma(ah[3], bh[3], -p[3]));
    la = fma(ah[1], bl[1], la);
    lb = fma(ah[3], bl[3], lb);
    la = fma(al[1], bh[1], la);
    lb = fma(al[3], bh[3], lb);
    float s01, r01, s23, r23, s, r;
    two_sum(p[0], p[1], s01, r01);
    two_sum(p[2], p[3], s23, r23);
    two_sum(s01, s23, s, r);
    const float lo = add(add(la, lb), add(add(r01, r23), r));
    fast_two_sum(s, lo, h, l);
#else
    float p[4], lo;
#pragma unroll
    for (int k = 0; k < 4; ++k) p[k] = mul(ah[k], bh[k]);
    lo = fma(ah[0], bh[0], -p[0]);
#pragma unroll
    for (int k = 1; k < 4; ++k) lo = add(lo, fma(ah[k], bh[k], -p[k]));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        lo = fma(ah[k], bl[k], lo);
        lo = fma(al[k], bh[k], lo);
    }
    float s, r;
    two_sum(p[0], p[1], s, r);
    lo = add(lo, r);
    two_sum(s, p[2], s, r);
    lo = add(lo, r);
    two_sum(s, p[3], s, r);
    lo = add(lo, r);
    fast_two_sum(s, lo, h, l);
#endif
}

// Sum of two terms a0*b0 + a1*b1, renormalised.
QS_HD void dot2(float a0h, float a0l, float b0h, float b0l, float a1h, float a1l, float b1h, float b1l, float &h,
                float &l) {
    const float p0 = mul(a0h, b0h), p1 = mul(a1h, b1h);
    float lo = add(fma(a0h, b0h, -p0), fma(a1h, b1h, -p1));
    lo = fma(a0h, b0l, lo);
    lo = fma(a0l, b0h, lo);
    lo = fma(a1h, b1l, lo);
    lo = fma(a1l, b1h, lo);
    float s, r;
    two_sum(p0, p1, s, r);
    lo = add(lo, r);
    fast_two_sum(s, lo, h, l);
}

// x + y and x - y for double-single x, y (the Hadamard butterfly).
QS_HD void add2(float xh, float xl, float yh, float yl, float &h, float &l) {
    float s, r;
    two_sum(xh, yh, s, r);
    r = add(r, add(xl, yl));
    fast_two_sum(s, r, h, l);
}

// x * c for double-single x and c.
QS_HD void mul1(float xh, float xl, float ch, float cl, float &h, float &l) {
    const float p = mul(xh, ch);
    float e = fma(xh, ch, -p);
    e = fma(xh, cl, e);
    e = fma(xl, ch, e);
    fast_two_sum(p, e, h, l);
}

// A complex double-single amplitude: re = (rh, rl), im = (ih, il).
struct camp {
    float rh, rl, ih, il;
};

// A complex double-single constant (matrix entry).
struct ccst {
    float rh, rl, ih, il;
};

// a*x + b*y (complex), the output of one row of a 2x2 update.
QS_HD camp cmad2(const ccst &a, const camp &x, const ccst &b, const camp &y) {
    camp o;
    {
        const float ah[4] = {a.rh, -a.ih, b.rh, -b.ih}, al[4] = {a.rl, -a.il, b.rl, -b.il};
        const float xh[4] = {x.rh, x.ih, y.rh, y.ih}, xl[4] = {x.rl, x.il, y.rl, y.il};
        dot4(ah, al, xh, xl, o.rh, o.rl);
    }
    {
        const float ah[4] = {a.rh, a.ih, b.rh, b.ih}, al[4] = {a.rl, a.il, b.rl, b.il};
        const float xh[4] = {x.ih, x.rh, y.ih, y.rh}, xl[4] = {x.il, x.rl, y.il, y.rl};
        dot4(ah, al, xh, xl, o.ih, o.il);
    }
    return o;
}

// a*x + b*y with real a, b (a.rh, a.rl and b.rh, b.rl; the imaginary parts
// are ignored): each output component is a two-term dot product.
QS_HD camp rmad2(const ccst &a, const camp &x, const ccst &b, const camp &y) {
    camp o;
    dot2(a.rh, a.rl, x.rh, x.rl, b.rh, b.rl, y.rh, y.rl, o.rh, o.rl);
    dot2(a.rh, a.rl, x.ih, x.il, b.rh, b.rl, y.ih, y.il, o.ih, o.il);
    return o;
}

// d*x (complex).
QS_HD camp cmul(const ccst &d, const camp &x) {
    camp o;
    dot2(d.rh, d.rl, x.rh, x.rl, -d.ih, -d.il, x.ih, x.il, o.rh, o.rl);
    dot2(d.rh, d.rl, x.ih, x.il, d.ih, d.il, x.rh, x.rl, o.ih, o.il);
    return o;
}

// Hadamard butterfly without its factor: (x + y, x - y).
QS_HD void butterfly(camp &x, camp &y) {
    camp s, d;
    add2(x.rh, x.rl, y.rh, y.rl, s.rh, s.rl);
    add2(x.ih, x.il, y.ih, y.il, s.ih, s.il);
    add2(x.rh, x.rl, -y.rh, -y.rl, d.rh, d.rl);
    add2(x.ih, x.il, -y.ih, -y.il, d.ih, d.il);
    x = s;
    y = d;
}

QS_HD camp load(double re, double im) {
    camp a;
    split(re, a.rh, a.rl);
    split(im, a.ih, a.il);
    return a;
}

// Splits a double constant exactly as far as 48 bits reach (rounded to
// nearest at the second float): h = fl(c), l = fl(c - h).  Host-side, for
// matrix entries.
inline void split_const(double c, float &h, float &l) {
    h = float(c);
    l = float(c - double(h));
}

}  // namespace ds
}  // namespace qs
