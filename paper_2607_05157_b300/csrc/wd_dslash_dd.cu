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
// near either).
//
// The stencil input is a field in the double-float layout ("ddl"): the FP64
// eo layout with each complex double2 replaced by the float4
// (re.h, im.h, re.l, im.l) -- same 16 bytes, same indexing.  An FP64 input is
// split once by the memory-bound pass k_to_ddl instead of once per
// neighbour read (8 times) inside the stencil; the intermediate field of the
// two-hop Schur residual is written in ddl directly.  The addend w is FP64,
// w2 FP64 or ddl (A.w2_ddl); the output is FP64 (h + l, one FP64 add) or ddl.
//
// Two arithmetic variants: scalar (R = 1, 2 RHS per thread) and packed
// (R code 11, 12): (re, im) pairs through the f32x2 FMA/ADD instructions,
// about half the FP32 instructions.
#include "wd_internal.h"
#include "wd_dd.cuh"
#include "wd_spin.cuh"

namespace wd {

// one site of a ddl field
__device__ __forceinline__ void load_dd(const void *p, long Vh, long s, cx<dd> v[12]) {
    const float4 *q = (const float4 *)p + s;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const float4 a = __ldg(q + k * Vh);
        v[k] = cmake(dd_make(a.x, a.z), dd_make(a.y, a.w));
    }
}

// FP64 eo field -> ddl (n complex numbers)
__global__ void k_to_ddl(const double2 *in, float4 *out, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const double2 v = __ldg(in + i);
        const dd a = d2dd(v.x), b = d2dd(v.y);
        out[i] = make_float4(a.h, b.h, a.l, b.l);
    }
}

cudaError_t launch_to_ddl(const void *in, void *out, long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long blocks = (n + 255) / 256;
    if (blocks > 148L * 16) blocks = 148L * 16;
    k_to_ddl<<<(unsigned)blocks, 256, 0, st>>>((const double2 *)in, (float4 *)out, n);
    return cudaGetLastError();
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

template <int R, bool DAG, bool OUTDD>
__global__ void __launch_bounds__(128) hop_kernel_dd(HopArgs A) {
    const int rb = blockIdx.x % A.nrb;
    const int s = (blockIdx.x / A.nrb) * blockDim.x + threadIdx.x;
    if (s >= A.g.Vh || tile_rhs(A, rb, 0, R) < 0) return;
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
            const int rhs = tile_rhs(A, rb, r, R);
            if (rhs >= 0 && hop_reaches(A, rhs, t)) {
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
        const int rhs = tile_rhs(A, rb, r, R);
        if (rhs < 0) break;
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
        if (A.w2 && A.w2_ddl) {
            const float4 *q = (const float4 *)A.w2 + (size_t)rhs * 12 * Vh + s;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const float4 v = __ldg(q + k * Vh);
                o[k].re = o[k].re + dd_mul(c, dd_make(v.x, v.z));
                o[k].im = o[k].im + dd_mul(c, dd_make(v.y, v.w));
            }
        } else if (A.w2) {
            const double2 *q = (const double2 *)A.w2 + (size_t)rhs * 12 * Vh + s;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const double2 v = __ldg(q + k * Vh);
                o[k].re = o[k].re + dd_mul(c, d2dd(v.x));
                o[k].im = o[k].im + dd_mul(c, d2dd(v.y));
            }
        }
        if constexpr (OUTDD) {
            float4 *q = (float4 *)A.out + (size_t)rhs * 12 * Vh + s;
#pragma unroll
            for (int k = 0; k < 12; ++k) q[k * Vh] = make_float4(o[k].re.h, o[k].im.h, o[k].re.l, o[k].im.l);
        } else {
            double2 *q = (double2 *)A.out + (size_t)rhs * 12 * Vh + s;
#pragma unroll
            for (int k = 0; k < 12; ++k) q[k * Vh] = make_double2(dd2d(o[k].re), dd2d(o[k].im));
        }
    }
}

// ---- packed variant: a complex double-float number as two FP32 pairs --------
// zdd: h = (re.h, im.h), l = (re.l, im.l); every operation below acts on the
// real and imaginary parts at once through the f32x2 instructions.
struct zdd { float2 h, l; };

__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 swp(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// a - b, exactly rounded (one FMA with -1)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, mk2(-1.f, -1.f), a); }

// a + sg*(bh + bl), sg a pair of +-1: TwoSum on the high parts with the sign
// folded in (nbv = a - s is the negated "virtual b" of the TwoSum)
__device__ __forceinline__ zdd zadd(const zdd &a, float2 bh, float2 bl, float2 sg) {
    const float2 s = __ffma2_rn(bh, sg, a.h);
    const float2 nbv = sub2(a.h, s);
    const float2 av = __fadd2_rn(s, nbv);
    const float2 e = __fadd2_rn(sub2(a.h, av), __ffma2_rn(bh, sg, nbv));
    zdd r;
    r.h = s;
    r.l = __ffma2_rn(bl, sg, __fadd2_rn(a.l, e));
    return r;
}

// (Ah + Al) * (Bh + Bl) elementwise; nBh = -Bh
__device__ __forceinline__ zdd zmul(float2 Ah, float2 Al, float2 Bh, float2 nBh, float2 Bl) {
    const float2 p = __fmul2_rn(Ah, Bh), np = __fmul2_rn(Ah, nBh);
    float2 x = __ffma2_rn(Ah, Bh, np);          // exact error of p
    x = __ffma2_rn(Ah, Bl, x);
    x = __ffma2_rn(Al, Bh, x);
    zdd r;
    r.h = p;
    r.l = x;
    return r;
}

// acc += (Ah + Al) * (Bh + Bl) elementwise; nBh = -Bh
__device__ __forceinline__ void zfma(zdd &acc, float2 Ah, float2 Al, float2 Bh, float2 nBh, float2 Bl) {
    const float2 np = __fmul2_rn(Ah, nBh);      // -p
    float2 x = __ffma2_rn(Ah, Bh, np);          // exact error of p
    x = __ffma2_rn(Ah, Bl, x);
    x = __ffma2_rn(Al, Bh, x);
    const float2 s = sub2(acc.h, np);           // acc.h + p
    const float2 nbv = sub2(acc.h, s);
    const float2 av = __fadd2_rn(s, nbv);
    const float2 e = __fadd2_rn(sub2(acc.h, av), sub2(nbv, np));
    acc.h = s;
    acc.l = __fadd2_rn(acc.l, __fadd2_rn(x, e));
}

// spin projection and reconstruction: the sign tables of the FP32 packed
// stencil, with the TwoSum additions above
template <int MU, int S>
__device__ __forceinline__ void proj_z(const zdd p[12], zdd h[6]) {
    const float s = (float)S;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const zdd p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
        if (MU == 0) {        // A = -i s1: (-i p3, -i p2)
            h[c] = zadd(p0, swp(p3.h), swp(p3.l), mk2(s, -s));
            h[3 + c] = zadd(p1, swp(p2.h), swp(p2.l), mk2(s, -s));
        } else if (MU == 1) { // A = -i s2: (-p3, p2)
            h[c] = zadd(p0, p3.h, p3.l, mk2(-s, -s));
            h[3 + c] = zadd(p1, p2.h, p2.l, mk2(s, s));
        } else if (MU == 2) { // A = -i s3: (-i p2, i p3)
            h[c] = zadd(p0, swp(p2.h), swp(p2.l), mk2(s, -s));
            h[3 + c] = zadd(p1, swp(p3.h), swp(p3.l), mk2(-s, s));
        } else {              // A = 1
            h[c] = zadd(p0, p2.h, p2.l, mk2(s, s));
            h[3 + c] = zadd(p1, p3.h, p3.l, mk2(s, s));
        }
    }
}

template <int MU, int S>
__device__ __forceinline__ void recon_z(zdd acc[12], const zdd h[6]) {
    const float s = (float)S;
    const float2 one = mk2(1.f, 1.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const zdd h0 = h[c], h1 = h[3 + c];
        acc[c] = zadd(acc[c], h0.h, h0.l, one);
        acc[3 + c] = zadd(acc[3 + c], h1.h, h1.l, one);
        if (MU == 0) {        // A^dag (h0, h1) = (i h1, i h0)
            acc[6 + c] = zadd(acc[6 + c], swp(h1.h), swp(h1.l), mk2(-s, s));
            acc[9 + c] = zadd(acc[9 + c], swp(h0.h), swp(h0.l), mk2(-s, s));
        } else if (MU == 1) { // (h1, -h0)
            acc[6 + c] = zadd(acc[6 + c], h1.h, h1.l, mk2(s, s));
            acc[9 + c] = zadd(acc[9 + c], h0.h, h0.l, mk2(-s, -s));
        } else if (MU == 2) { // (i h0, -i h1)
            acc[6 + c] = zadd(acc[6 + c], swp(h0.h), swp(h0.l), mk2(-s, s));
            acc[9 + c] = zadd(acc[9 + c], swp(h1.h), swp(h1.l), mk2(s, -s));
        } else {              // (h0, h1)
            acc[6 + c] = zadd(acc[6 + c], h0.h, h0.l, mk2(s, s));
            acc[9 + c] = zadd(acc[9 + c], h1.h, h1.l, mk2(s, s));
        }
    }
}

template <bool DAG>
__device__ __forceinline__ void project_dir_z(int d, const zdd psi[12], zdd h[6]) {
    constexpr int F = DAG ? +1 : -1, B = -F;
    switch (d) {
        case 0: proj_z<0, F>(psi, h); break;
        case 1: proj_z<1, F>(psi, h); break;
        case 2: proj_z<2, F>(psi, h); break;
        case 3: proj_z<3, F>(psi, h); break;
        case 4: proj_z<0, B>(psi, h); break;
        case 5: proj_z<1, B>(psi, h); break;
        case 6: proj_z<2, B>(psi, h); break;
        default: proj_z<3, B>(psi, h); break;
    }
}

template <bool DAG>
__device__ __forceinline__ void reconstruct_dir_z(int d, zdd acc[12], const zdd uh[6]) {
    constexpr int F = DAG ? +1 : -1, B = -F;
    switch (d) {
        case 0: recon_z<0, F>(acc, uh); break;
        case 1: recon_z<1, F>(acc, uh); break;
        case 2: recon_z<2, F>(acc, uh); break;
        case 3: recon_z<3, F>(acc, uh); break;
        case 4: recon_z<0, B>(acc, uh); break;
        case 5: recon_z<1, B>(acc, uh); break;
        case 6: recon_z<2, B>(acc, uh); break;
        default: recon_z<3, B>(acc, uh); break;
    }
}

// out[3sp+i] = sum_j u[3i+j] h[3sp+j]; u[k] = (re.h, im.h, re.l, im.l).  Each
// complex product is (re, re) * (h.re, h.im) + (-im, im) * (h.im, h.re).
__device__ __forceinline__ void su3_z(const float4 u[9], const zdd h[6], zdd out[6]) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            zdd a;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float4 uu = u[3 * i + j];
                const zdd hj = h[3 * sp + j];
                const float2 nh = neg2(hj.h), sh = swp(hj.h);
                if (j == 0) a = zmul(mk2(uu.x, uu.x), mk2(uu.z, uu.z), hj.h, nh, hj.l);
                else zfma(a, mk2(uu.x, uu.x), mk2(uu.z, uu.z), hj.h, nh, hj.l);
                zfma(a, mk2(-uu.y, uu.y), mk2(-uu.w, uu.w), sh, swp(nh), swp(hj.l));
            }
            out[3 * sp + i] = a;
        }
}

template <int R, bool DAG, bool OUTDD>
__global__ void __launch_bounds__(128) hop_kernel_ddz(HopArgs A) {
    const int rb = blockIdx.x % A.nrb;
    const int s = (blockIdx.x / A.nrb) * blockDim.x + threadIdx.x;
    if (s >= A.g.Vh || tile_rhs(A, rb, 0, R) < 0) return;
    const Geom &g = A.g;
    int x, y, z, t;
    eo_coords(g, A.p, s, x, y, z, t);
    const long Vh = g.Vh;

    zdd acc[R][12];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) { acc[r][k].h = mk2(0.f, 0.f); acc[r][k].l = mk2(0.f, 0.f); }

#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
        const int mu = d & 3;
        int c[4] = {x, y, z, t};
        const int L[4] = {g.X, g.Y, g.Z, g.T};
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (m == mu) c[m] = d < 4 ? (c[m] + 1 == L[m] ? 0 : c[m] + 1) : (c[m] == 0 ? L[m] - 1 : c[m] - 1);
        const int nb = eo_index(g, c[0], c[1], c[2], c[3]);
        float4 u[9];
        {
            const float2 *qh = (const float2 *)A.gauge + (size_t)d * 9 * Vh + s;
            const float2 *ql = (const float2 *)A.gauge_lo + (size_t)d * 9 * Vh + s;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float2 h = __ldg(qh + k * Vh), l = __ldg(ql + k * Vh);
                u[k] = make_float4(h.x, h.y, l.x, l.y);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int rhs = tile_rhs(A, rb, r, R);
            if (rhs >= 0 && hop_reaches(A, rhs, t)) {
                zdd psi[12], h[6], uh[6];
                const float4 *q = (const float4 *)A.in + (size_t)rhs * 12 * Vh + nb;
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    const float4 a = __ldg(q + k * Vh);
                    psi[k].h = mk2(a.x, a.y);
                    psi[k].l = mk2(a.z, a.w);
                }
                project_dir_z<DAG>(d, psi, h);
                su3_z(u, h, uh);
                reconstruct_dir_z<DAG>(d, acc[r], uh);
            }
        }
    }

    const dd a = d2dd(A.a), b = d2dd(A.b), c = d2dd(A.c);
    const float2 ah = mk2(a.h, a.h), al = mk2(a.l, a.l), bh = mk2(b.h, b.h), bl = mk2(b.l, b.l);
    const float2 ch = mk2(c.h, c.h), cl = mk2(c.l, c.l);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int rhs = tile_rhs(A, rb, r, R);
        if (rhs < 0) break;
        zdd o[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) o[k] = zmul(bh, bl, acc[r][k].h, neg2(acc[r][k].h), acc[r][k].l);
        if (A.w) {
            const double2 *q = (const double2 *)A.w + (size_t)rhs * 12 * Vh + s;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const double2 v = __ldg(q + k * Vh);
                const dd vr = d2dd(v.x), vi = d2dd(v.y);
                const float2 wh = mk2(vr.h, vi.h);
                zfma(o[k], ah, al, wh, neg2(wh), mk2(vr.l, vi.l));
            }
        }
        if (A.w2 && A.w2_ddl) {
            const float4 *q = (const float4 *)A.w2 + (size_t)rhs * 12 * Vh + s;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const float4 v = __ldg(q + k * Vh);
                const float2 wh = mk2(v.x, v.y);
                zfma(o[k], ch, cl, wh, neg2(wh), mk2(v.z, v.w));
            }
        } else if (A.w2) {
            const double2 *q = (const double2 *)A.w2 + (size_t)rhs * 12 * Vh + s;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const double2 v = __ldg(q + k * Vh);
                const dd vr = d2dd(v.x), vi = d2dd(v.y);
                const float2 wh = mk2(vr.h, vi.h);
                zfma(o[k], ch, cl, wh, neg2(wh), mk2(vr.l, vi.l));
            }
        }
        if constexpr (OUTDD) {
            float4 *q = (float4 *)A.out + (size_t)rhs * 12 * Vh + s;
#pragma unroll
            for (int k = 0; k < 12; ++k) q[k * Vh] = make_float4(o[k].h.x, o[k].h.y, o[k].l.x, o[k].l.y);
        } else {
            double2 *q = (double2 *)A.out + (size_t)rhs * 12 * Vh + s;
#pragma unroll
            for (int k = 0; k < 12; ++k)
                q[k * Vh] = make_double2(dd2d(dd_make(o[k].h.x, o[k].l.x)), dd2d(dd_make(o[k].h.y, o[k].l.y)));
        }
    }
}

// R = 1, 2: scalar double-float; R = 11, 12: packed.  A.in is a ddl field.
cudaError_t launch_hop_dd(const HopArgs &A0, int R, bool dag, int threads, bool out_dd, cudaStream_t st) {
    HopArgs A = A0;
    if (A.nrhs <= 0) return cudaSuccess;
    const bool packed = R > 10;
    int RR = packed ? R - 10 : R;
    if (RR != 1 && RR != 2) RR = 1;
    if (threads > 128) threads = 128;
    A.nrb = (A.nrhs + RR - 1) / RR;
    const int sblocks = (A.g.Vh + threads - 1) / threads;
    const dim3 grid((unsigned)(sblocks * A.nrb));
#define WD_DD_CASE(K, RV)                                                                            \
    if (RR == RV) {                                                                                  \
        if (dag) { if (out_dd) K<RV, true, true><<<grid, threads, 0, st>>>(A);                       \
                   else K<RV, true, false><<<grid, threads, 0, st>>>(A); }                          \
        else { if (out_dd) K<RV, false, true><<<grid, threads, 0, st>>>(A);                          \
               else K<RV, false, false><<<grid, threads, 0, st>>>(A); }                             \
    }
    if (packed) {
        WD_DD_CASE(hop_kernel_ddz, 1) WD_DD_CASE(hop_kernel_ddz, 2)
    } else {
        WD_DD_CASE(hop_kernel_dd, 1) WD_DD_CASE(hop_kernel_dd, 2)
    }
#undef WD_DD_CASE
    return cudaGetLastError();
}

}  // namespace wd
