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

// The eight directions run as one rolled loop: the SU(3) product and the input
// conversion (most of the instructions) exist once in the code, only the spin
// projection and reconstruction are specialised per direction behind a
// warp-uniform switch.  Unrolled, the directions make ~11k instructions of
// straight-line double-float code and the kernel stalls on instruction fetch.
template <bool DAG>
__device__ __forceinline__ void project_dir(int d, const cx<dd> psi[12], cx<dd> h[6]) {
    // D uses (1 - g) forward and (1 + g) backward; D^dag swaps them
    constexpr int F = DAG ? +1 : -1, B = -F;
    switch (d) {
        case 0: spin_project<0, F>(psi, h); break;
        case 1: spin_project<1, F>(psi, h); break;
        case 2: spin_project<2, F>(psi, h); break;
        case 3: spin_project<3, F>(psi, h); break;
        case 4: spin_project<0, B>(psi, h); break;
        case 5: spin_project<1, B>(psi, h); break;
        case 6: spin_project<2, B>(psi, h); break;
        default: spin_project<3, B>(psi, h); break;
    }
}

template <bool DAG>
__device__ __forceinline__ void reconstruct_dir(int d, cx<dd> acc[12], const cx<dd> uh[6]) {
    constexpr int F = DAG ? +1 : -1, B = -F;
    switch (d) {
        case 0: spin_reconstruct_add<0, F>(acc, uh); break;
        case 1: spin_reconstruct_add<1, F>(acc, uh); break;
        case 2: spin_reconstruct_add<2, F>(acc, uh); break;
        case 3: spin_reconstruct_add<3, F>(acc, uh); break;
        case 4: spin_reconstruct_add<0, B>(acc, uh); break;
        case 5: spin_reconstruct_add<1, B>(acc, uh); break;
        case 6: spin_reconstruct_add<2, B>(acc, uh); break;
        default: spin_reconstruct_add<3, B>(acc, uh); break;
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

    cx<dd> acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = cmake(dd_make(0.f, 0.f), dd_make(0.f, 0.f));

#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
        // neighbour x + mu (d < 4) or x - mu (d >= 4) with periodic wrap (the
        // boundary factor is folded into the links)
        const int mu = d & 3;
        int c[4] = {x, y, z, t};
        const int L[4] = {g.X, g.Y, g.Z, g.T};
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (m == mu) c[m] = d < 4 ? (c[m] + 1 == L[m] ? 0 : c[m] + 1) : (c[m] == 0 ? L[m] - 1 : c[m] - 1);
        const int nb = eo_index(g, c[0], c[1], c[2], c[3]);
        const long Vh = g.Vh;
        cx<dd> u[9];
        {
            const float2 *qh = (const float2 *)A.gauge + (size_t)d * 9 * Vh + s;
            const float2 *ql = (const float2 *)A.gauge_lo + (size_t)d * 9 * Vh + s;
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
                project_dir<DAG>(d, psi, h);
                su3_dd(u, h, uh);
                reconstruct_dir<DAG>(d, acc[r], uh);
            }
        }
    }

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
