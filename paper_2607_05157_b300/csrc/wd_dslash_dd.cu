// Fine Wilson hopping stencil on FP64 fields with double-float arithmetic.
//
// Same operation as the FP64 stencil (out = a*w + c*w2 + b*H(in), H the
// hopping term of the Wilson-Dirac operator of Sec. 1), for the FP64 steps of
// the mixed-precision solves: the Schur source, the defect-correction residual
// and the odd-site reconstruction.  B300 issues FP64 at about 1/64 of its
// FP32 rate, so the FP64 stencil is bound by FP64 arithmetic long before
// memory.  Here every real is carried as an unevaluated pair of FP32 numbers
// v = h + l ("double-float"):
//   * FP64 inputs are split exactly into the top 24 significant bits (h, by
//     truncation) and the next 23 (l) with integer operations only;
//   * the links are the FP32 copy (h) plus a stored FP32 remainder (l);
//   * products use the error-free transformation p + e = a.h * b.h (one FMA
//     gives e exactly), the cross terms a.h*b.l + a.l*b.h in plain FP32;
//   * sums use Knuth's TwoSum on the high parts, the low parts in plain FP32.
// The result agrees with the FP64 stencil normwise to about 2^-44 (the
// split keeps 47 bits; each product and sum loses at most 2^-48 relative to
// the magnitudes involved).  Inputs below 2^-103 in magnitude are treated as
// zero and inputs of 2^128 or more as NaN (no field the solver meets comes
// near either).  Outputs are written as FP64 (h + l, one FP64 add).
#include "wd_internal.h"
#include "wd_spin.cuh"

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

__device__ __forceinline__ void load_dd(const void *p, long Vh, long s, cx<dd> v[12]) {
    const double2 *q = (const double2 *)p + s;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 a = __ldg(q + k * Vh);
        v[k] = cmake(d2dd(a.x), d2dd(a.y));
    }
}

// out[3s+i] = sum_j u[3i+j] in[3s+j], s = 0, 1
__device__ __forceinline__ void su3_dd(const cx<dd> u[9], const cx<dd> in[6], cx<dd> out[6]) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const cx<dd> u0 = u[3 * i], h0 = in[3 * s];
            dd re = dd_mul(u0.re, h0.re), im = dd_mul(u0.re, h0.im);
            dd_fma(re, -u0.im, h0.im);
            dd_fma(im, u0.im, h0.re);
#pragma unroll
            for (int j = 1; j < 3; ++j) {
                const cx<dd> uj = u[3 * i + j], hj = in[3 * s + j];
                dd_fma(re, uj.re, hj.re);
                dd_fma(re, -uj.im, hj.im);
                dd_fma(im, uj.re, hj.im);
                dd_fma(im, uj.im, hj.re);
            }
            out[3 * s + i] = cmake(re, im);
        }
}

template <int R, int D, bool DAG>
__device__ __forceinline__ void hop_dir_dd(const HopArgs &A, int s, int nb, int rb, cx<dd> acc[][12]) {
    constexpr int MU = D & 3;
    constexpr bool FWD = D < 4;
    constexpr int SIGN = (FWD != DAG) ? -1 : +1;
    const long Vh = A.g.Vh;
    cx<dd> u[9];
    {
        const float2 *qh = (const float2 *)A.gauge + (size_t)D * 9 * Vh + s;
        const float2 *ql = (const float2 *)A.gauge_lo + (size_t)D * 9 * Vh + s;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float2 h = __ldg(qh + k * Vh), l = __ldg(ql + k * Vh);
            u[k] = cmake(dd_make(h.x, l.x), dd_make(h.y, l.y));
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int rhs = rb * R + r;
        if (rhs < A.nrhs) {
            cx<dd> psi[12], h[6], uh[6];
            load_dd((const double2 *)A.in + (size_t)rhs * 12 * Vh, Vh, nb, psi);
            spin_project<MU, SIGN>(psi, h);
            su3_dd(u, h, uh);
            spin_reconstruct_add<MU, SIGN>(acc[r], uh);
        }
    }
}

template <int R, bool DAG>
__global__ void __launch_bounds__(128) hop_kernel_dd(HopArgs A) {
    const int rb = blockIdx.x % A.nrb;
    const int s = (blockIdx.x / A.nrb) * blockDim.x + threadIdx.x;
    if (s >= A.g.Vh) return;
    const Geom &g = A.g;
    int x, y, z, t;
    eo_coords(g, A.p, s, x, y, z, t);
    const int xp = x + 1 == g.X ? 0 : x + 1, xm = x == 0 ? g.X - 1 : x - 1;
    const int yp = y + 1 == g.Y ? 0 : y + 1, ym = y == 0 ? g.Y - 1 : y - 1;
    const int zp = z + 1 == g.Z ? 0 : z + 1, zm = z == 0 ? g.Z - 1 : z - 1;
    const int tp = t + 1 == g.T ? 0 : t + 1, tm = t == 0 ? g.T - 1 : t - 1;

    cx<dd> acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = cmake(dd_make(0.f, 0.f), dd_make(0.f, 0.f));

    hop_dir_dd<R, 0, DAG>(A, s, eo_index(g, xp, y, z, t), rb, acc);
    hop_dir_dd<R, 1, DAG>(A, s, eo_index(g, x, yp, z, t), rb, acc);
    hop_dir_dd<R, 2, DAG>(A, s, eo_index(g, x, y, zp, t), rb, acc);
    hop_dir_dd<R, 3, DAG>(A, s, eo_index(g, x, y, z, tp), rb, acc);
    hop_dir_dd<R, 4, DAG>(A, s, eo_index(g, xm, y, z, t), rb, acc);
    hop_dir_dd<R, 5, DAG>(A, s, eo_index(g, x, ym, z, t), rb, acc);
    hop_dir_dd<R, 6, DAG>(A, s, eo_index(g, x, y, zm, t), rb, acc);
    hop_dir_dd<R, 7, DAG>(A, s, eo_index(g, x, y, z, tm), rb, acc);

    const long Vh = g.Vh;
    const dd a = d2dd(A.a), b = d2dd(A.b), c = d2dd(A.c);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int rhs = rb * R + r;
        if (rhs >= A.nrhs) break;
        cx<dd> o[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = cmake(dd_mul(b, acc[r][k].re), dd_mul(b, acc[r][k].im));
        if (A.w) {
            const double2 *q = (const double2 *)A.w + (size_t)rhs * 12 * Vh + s;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const double2 v = __ldg(q + k * Vh);
                o[k].re = o[k].re + dd_mul(a, d2dd(v.x));
                o[k].im = o[k].im + dd_mul(a, d2dd(v.y));
            }
        }
        if (A.w2) {
            const double2 *q = (const double2 *)A.w2 + (size_t)rhs * 12 * Vh + s;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const double2 v = __ldg(q + k * Vh);
                o[k].re = o[k].re + dd_mul(c, d2dd(v.x));
                o[k].im = o[k].im + dd_mul(c, d2dd(v.y));
            }
        }
        double2 *q = (double2 *)A.out + (size_t)rhs * 12 * Vh + s;
#pragma unroll
        for (int k = 0; k < 12; ++k) q[k * Vh] = make_double2(dd2d(o[k].re), dd2d(o[k].im));
    }
}

cudaError_t launch_hop_dd(const HopArgs &A0, int R, bool dag, int threads, cudaStream_t st) {
    HopArgs A = A0;
    if (A.nrhs <= 0) return cudaSuccess;
    if (R != 1 && R != 2) R = 1;
    if (threads > 128) threads = 128;
    A.nrb = (A.nrhs + R - 1) / R;
    const int sblocks = (A.g.Vh + threads - 1) / threads;
    const dim3 grid((unsigned)(sblocks * A.nrb));
    if (R == 1) {
        if (dag) hop_kernel_dd<1, true><<<grid, threads, 0, st>>>(A);
        else hop_kernel_dd<1, false><<<grid, threads, 0, st>>>(A);
    } else {
        if (dag) hop_kernel_dd<2, true><<<grid, threads, 0, st>>>(A);
        else hop_kernel_dd<2, false><<<grid, threads, 0, st>>>(A);
    }
    return cudaGetLastError();
}

}  // namespace wd
