// Scalar double-float ("dd") arithmetic: a real carried as an unevaluated
// pair of FP32 numbers h + l, for the FP64 steps of the mixed-precision
// solves on a GPU whose FP64 rate is a small fraction of its FP32 rate.
// Products keep the exact FMA error of the high parts plus the cross terms;
// sums use Knuth's TwoSum on the high parts and plain FP32 on the low parts.
#pragma once
#include <cuda_runtime.h>

namespace wd {

struct dd { float h, l; };

__device__ __forceinline__ dd dd_make(float h, float l) { dd r; r.h = h; r.l = l; return r; }
__device__ __forceinline__ dd operator-(dd a) { return dd_make(-a.h, -a.l); }

// s + e == a + b exactly (Knuth's TwoSum; no ordering assumption)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

__device__ __forceinline__ dd operator+(dd a, dd b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    return dd_make(s, __fadd_rn(__fadd_rn(a.l, b.l), e));
}
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }

// a * b as an unevaluated pair (p, x): p = fl(a.h b.h), x = its exact error
// plus the cross terms.
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
    const float p = __fmul_rn(a.h, b.h);
    float x = __fmaf_rn(a.h, b.h, -p);
    x = __fmaf_rn(a.h, b.l, x);
    x = __fmaf_rn(a.l, b.h, x);
    return dd_make(p, x);
}

// acc += a * b
__device__ __forceinline__ void dd_fma(dd &acc, dd a, dd b) {
    const dd q = dd_mul(a, b);
    float s, t;
    two_sum(acc.h, q.h, s, t);
    acc = dd_make(s, __fadd_rn(acc.l, __fadd_rn(q.l, t)));
}

// FP64 -> (h, l) with integer operations: h = the top 24 significant bits
// (round toward zero, exponent rebiased 1023 -> 127), l = the next 23 bits,
// formed as (2^k (1 + m/2^23)) - 2^k, an exact FP32 subtraction.
__device__ __forceinline__ dd d2dd(double d) {
    const unsigned H = (unsigned)__double2hiint(d), L = (unsigned)__double2loint(d);
    const unsigned sgn = H & 0x80000000u;
    const unsigned t = __funnelshift_l(L, H, 3);                          // exponent mod 512 | top 23 bits
    const unsigned hb = ((t + 0x40000000u) & 0x7fffffffu) | sgn;          // exponent - 896
    const unsigned bb = (((t & 0xff800000u) - 0xCB800000u) & 0x7fffffffu) | sgn;   // exponent - 919
    const unsigned ab = bb | ((L >> 6) & 0x007fffffu);
    const float lo = __fsub_rn(__uint_as_float(ab), __uint_as_float(bb));
    const unsigned mag = H & 0x7fffffffu;
    const bool ok = mag >= (920u << 20), big = mag >= (1151u << 20);
    const float hi = big ? __uint_as_float(0x7fc00000u) : (ok ? __uint_as_float(hb) : 0.f);
    return dd_make(hi, ok ? lo : 0.f);
}

__device__ __forceinline__ double dd2d(dd a) { return __dadd_rn((double)a.h, (double)a.l); }

}  // namespace wd
