// Shared device types for libwd: complex arithmetic, storage traits for the
// even-odd multi-RHS field layout, lattice geometry and error plumbing.
//
// Internal field layout ("eo layout"): one parity of an nrhs-field is
//   [rhs][chunk][Vh] of 16-byte chunks, Vh = V/2 sites of that parity,
// a site's 12 complex spin-colour components (index 3*spin + colour) spread
// over NCH chunks: 12 x double2 (FP64), 6 x float4 (FP32), 3 x 8 bf16 (BF16).
// A warp of consecutive sites reads each chunk as one contiguous 512-byte
// segment, so every spinor load is a fully coalesced 128-bit load.
// Links: [parity][dir 0..7][9][Vh] of complex pairs; dir mu < 4 holds
// U_mu(x), dir 4+mu holds U_mu(x-mu)^dag, both with the boundary factor
// folded in, so both hops read their links with unit stride.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace wd {

typedef __nv_bfloat16 bf16;

template <typename R> struct cx { R re, im; };

template <typename R> __device__ __forceinline__ cx<R> cmake(R a, R b) { cx<R> c; c.re = a; c.im = b; return c; }
template <typename R> __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return cmake(a.re + b.re, a.im + b.im); }
template <typename R> __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return cmake(a.re - b.re, a.im - b.im); }
template <typename R> __device__ __forceinline__ cx<R> operator*(R s, cx<R> a) { return cmake(s * a.re, s * a.im); }
// i*a and -i*a
template <typename R> __device__ __forceinline__ cx<R> times_i(cx<R> a) { return cmake(-a.im, a.re); }
template <typename R> __device__ __forceinline__ cx<R> times_mi(cx<R> a) { return cmake(a.im, -a.re); }
template <typename R> __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
    return cmake(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// acc += a * b
template <typename R> __device__ __forceinline__ void cfma(cx<R> &acc, cx<R> a, cx<R> b) {
    acc.re = fma(a.re, b.re, acc.re); acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im); acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R> __device__ __forceinline__ void cfma_conj(cx<R> &acc, cx<R> a, cx<R> b) {
    acc.re = fma(a.re, b.re, acc.re); acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im); acc.im = fma(-a.im, b.re, acc.im);
}

// ---- storage traits ------------------------------------------------------
// SIO<S>: a site's 12 complex components from/to the chunked eo layout.
// `p` points at the first chunk of one RHS of one parity; chunk k of site s
// is at p[k*Vh + s] (in 16-byte units).
template <typename S> struct SIO;

template <> struct SIO<double> {
    typedef double real;
    static constexpr int NCH = 12;
    __device__ __forceinline__ static void load(const void *p, long Vh, long s, cx<double> v[12]) {
        const double2 *q = (const double2 *)p + s;
#pragma unroll
        for (int k = 0; k < 12; ++k) { double2 a = __ldg(q + k * Vh); v[k] = cmake(a.x, a.y); }
    }
    __device__ __forceinline__ static void store(void *p, long Vh, long s, const cx<double> v[12]) {
        double2 *q = (double2 *)p + s;
#pragma unroll
        for (int k = 0; k < 12; ++k) q[k * Vh] = make_double2(v[k].re, v[k].im);
    }
};

template <> struct SIO<float> {
    typedef float real;
    static constexpr int NCH = 6;
    __device__ __forceinline__ static void load(const void *p, long Vh, long s, cx<float> v[12]) {
        const float4 *q = (const float4 *)p + s;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 a = __ldg(q + k * Vh);
            v[2 * k] = cmake(a.x, a.y); v[2 * k + 1] = cmake(a.z, a.w);
        }
    }
    __device__ __forceinline__ static void store(void *p, long Vh, long s, const cx<float> v[12]) {
        float4 *q = (float4 *)p + s;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            q[k * Vh] = make_float4(v[2 * k].re, v[2 * k].im, v[2 * k + 1].re, v[2 * k + 1].im);
    }
};

template <> struct SIO<bf16> {
    typedef float real;
    static constexpr int NCH = 3;
    __device__ __forceinline__ static void load(const void *p, long Vh, long s, cx<float> v[12]) {
        const uint4 *q = (const uint4 *)p + s;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 a = __ldg(q + k * Vh);
            const __nv_bfloat162 *h = (const __nv_bfloat162 *)&a;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float2 f = __bfloat1622float2(h[j]);
                v[4 * k + j] = cmake(f.x, f.y);
            }
        }
    }
    __device__ __forceinline__ static void store(void *p, long Vh, long s, const cx<float> v[12]) {
        uint4 *q = (uint4 *)p + s;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 a;
            __nv_bfloat162 *h = (__nv_bfloat162 *)&a;
#pragma unroll
            for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(v[4 * k + j].re, v[4 * k + j].im);
            q[k * Vh] = a;
        }
    }
};

// Compute type for a storage type: FP64 stays FP64, FP32 and BF16 compute in FP32.
template <typename S> struct RealOf { typedef typename SIO<S>::real type; };

// LIO<G>: one link (9 complex, row-major a*3+b) from [9][Vh] complex pairs.
template <typename G> struct LIO;
template <> struct LIO<double> {
    typedef double real;
    static constexpr int ELEM = 16;
    __device__ __forceinline__ static void load(const void *p, long Vh, long s, cx<double> u[9]) {
        const double2 *q = (const double2 *)p + s;
#pragma unroll
        for (int k = 0; k < 9; ++k) { double2 a = __ldg(q + k * Vh); u[k] = cmake(a.x, a.y); }
    }
};
template <> struct LIO<float> {
    typedef float real;
    static constexpr int ELEM = 8;
    __device__ __forceinline__ static void load(const void *p, long Vh, long s, cx<float> u[9]) {
        const float2 *q = (const float2 *)p + s;
#pragma unroll
        for (int k = 0; k < 9; ++k) { float2 a = __ldg(q + k * Vh); u[k] = cmake(a.x, a.y); }
    }
};
template <> struct LIO<bf16> {
    typedef float real;
    static constexpr int ELEM = 4;
    __device__ __forceinline__ static void load(const void *p, long Vh, long s, cx<float> u[9]) {
        const __nv_bfloat162 *q = (const __nv_bfloat162 *)p + s;
#pragma unroll
        for (int k = 0; k < 9; ++k) { float2 a = __bfloat1622float2(q[k * Vh]); u[k] = cmake(a.x, a.y); }
    }
};

// ---- geometry ------------------------------------------------------------
struct Geom {
    int X, Y, Z, T;     // extents (all even)
    int Xh;             // X / 2
    int Vh;             // V / 2
    int V;
};

// Coordinates of half-site s of parity p.
__device__ __forceinline__ void eo_coords(const Geom &g, int p, int s, int &x, int &y, int &z, int &t) {
    int xh = s % g.Xh;
    int r = s / g.Xh;
    y = r % g.Y; r /= g.Y;
    z = r % g.Z;
    t = r / g.Z;
    x = 2 * xh + ((p + y + z + t) & 1);
}
__device__ __forceinline__ int eo_index(const Geom &g, int x, int y, int z, int t) {
    return (x + g.X * (y + g.Y * (z + g.Z * t))) >> 1;
}

}  // namespace wd
