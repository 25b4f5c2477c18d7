// Krylov BLAS-1 for many right-hand sides on eo fields: layout conversions,
// precision conversions, fused BiCGStab updates with their dot products,
// and deterministic two-stage reductions (per-block FP64 partials, then a
// fixed-order sum), so that every Krylov scalar is an FP64 number.
//
// Elementwise kernels that mix precisions work per (RHS, site) unit: a
// thread loads the 12 complex components of a site of each operand through
// the layout-aware loaders (the chunk packing differs per precision).
// Kernels whose operands share one precision stream each RHS as a flat run
// of 16-byte chunks.  The FP64 steps of the defect correction (norms, the
// residual's FP32 copy, the solution update) run on the FP32 pipes, on
// integer splits of FP64 values or on double-float pairs.
#include <algorithm>

#include "wd_internal.h"

namespace wd {

// Site-level access: unit u = (rhs, site) of a field, u = rhs*Vh + s.
// All elementwise kernels go through these layout-aware loaders, because the
// chunk packing (and so the flat element order) of the eo layout differs per
// precision.  FLAT selects the plain layout [rhs][unit][12 complex] used for
// coarse-grid vectors, whose element order is the same in every precision.
template <typename S, typename RT, bool FLAT = false>
__device__ __forceinline__ void ldsite(const void *b, long Vh, long u, cx<RT> v[12]) {
    typedef typename SIO<S>::real T;
    cx<T> t[12];
    if (FLAT) {
        SIO<S>::load((const uint4 *)b + u * SIO<S>::NCH, 1, 0, t);
    } else {
        const long rhs = u / Vh, s = u - rhs * Vh;
        SIO<S>::load((const uint4 *)b + rhs * SIO<S>::NCH * Vh, Vh, s, t);
    }
#pragma unroll
    for (int j = 0; j < 12; ++j) v[j] = cmake((RT)t[j].re, (RT)t[j].im);
}
template <typename S, typename RT, bool FLAT = false>
__device__ __forceinline__ void stsite(void *b, long Vh, long u, const cx<RT> v[12]) {
    typedef typename SIO<S>::real T;
    cx<T> t[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) t[j] = cmake((T)v[j].re, (T)v[j].im);
    if (FLAT) {
        SIO<S>::store((uint4 *)b + u * SIO<S>::NCH, 1, 0, t);
    } else {
        const long rhs = u / Vh, s = u - rhs * Vh;
        SIO<S>::store((uint4 *)b + rhs * SIO<S>::NCH * Vh, Vh, s, t);
    }
}
template <typename S> struct RT_of { typedef typename SIO<S>::real type; };

size_t field_bytes(const Geom &g, int prec, int nrhs) {
    return (size_t)nrhs * g.Vh * spinor_bytes(prec);
}

int reduction_bpr(long units, int nrhs) {
    // at most one wave of the light reduction kernels (7 resident CTAs of 256
    // threads per SM): a second, partial wave costs more than fewer, longer
    // CTAs; >= 1 unit per thread
    int want = (7 * 148) / (nrhs > 0 ? nrhs : 1);
    int maxb = (int)((units + 255) / 256);
    if (want > maxb) want = maxb;
    if (want < 1) want = 1;
    if (want > 256) want = 256;
    return want;
}

// ---- block reduction of NQ doubles; thread 0 writes part[(q*nrhs+rhs)*bpr+bx]
template <int NQ>
__device__ __forceinline__ void block_partials(double v[NQ], double *part, int nrhs, int bpr) {
    __shared__ double sh[NQ][32];
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) sh[q][wid] = v[q];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            double a = lane < nw ? sh[q][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane == 0) part[((size_t)q * nrhs + blockIdx.y) * bpr + blockIdx.x] = a;
        }
    }
}

__device__ __forceinline__ double sum_part(const double *part, int q, int rhs, int nrhs, int bpr) {
    const double *p = part + ((size_t)q * nrhs + rhs) * bpr;
    double a = 0.0;
    for (int i = 0; i < bpr; ++i) a += p[i];
    return a;
}

struct Range { long g0, g1; };
// units [g0, g1) of RHS blockIdx.y handled by block blockIdx.x (per = units per RHS)
__device__ __forceinline__ Range my_range(long per) {
    const long chunk = (per + gridDim.x - 1) / gridDim.x;
    Range r;
    r.g0 = (long)blockIdx.y * per + (long)blockIdx.x * chunk;
    long e = r.g0 + chunk, lim = (long)(blockIdx.y + 1) * per;
    r.g1 = e < lim ? e : lim;
    return r;
}

// ---- layout conversion user <-> eo ------------------------------------------
template <typename TU, typename S>
__global__ void k_user_to_eo(const TU *user, void *even, void *odd, int nrhs, Geom g) {
    typedef typename RealOf<S>::type RT;
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long n = (long)g.V * nrhs;
    if (i >= n) return;
    const int rhs = (int)(i / g.V), site = (int)(i % g.V);
    int x = site % g.X, r = site / g.X;
    int y = r % g.Y; r /= g.Y;
    int z = r % g.Z, t = r / g.Z;
    const int p = (x + y + z + t) & 1;
    const TU *src = user + 24 * i;
    cx<RT> v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = cmake((RT)src[2 * k], (RT)src[2 * k + 1]);
    constexpr int NCH = SIO<S>::NCH;
    void *f = p ? odd : even;
    SIO<S>::store((uint4 *)f + (size_t)rhs * NCH * g.Vh, g.Vh, site >> 1, v);
}

template <typename S, typename TU>
__global__ void k_eo_to_user(const void *even, const void *odd, TU *user, int nrhs, Geom g) {
    typedef typename RealOf<S>::type RT;
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long n = (long)g.V * nrhs;
    if (i >= n) return;
    const int rhs = (int)(i / g.V), site = (int)(i % g.V);
    int x = site % g.X, r = site / g.X;
    int y = r % g.Y; r /= g.Y;
    int z = r % g.Z, t = r / g.Z;
    const int p = (x + y + z + t) & 1;
    constexpr int NCH = SIO<S>::NCH;
    const void *f = p ? odd : even;
    cx<RT> v[12];
    SIO<S>::load((const uint4 *)f + (size_t)rhs * NCH * g.Vh, g.Vh, site >> 1, v);
    TU *dst = user + 24 * i;
#pragma unroll
    for (int k = 0; k < 12; ++k) { dst[2 * k] = (TU)v[k].re; dst[2 * k + 1] = (TU)v[k].im; }
}

#define WD_DISPATCH_PREC(prec, S, ...)                         \
    do {                                                       \
        if ((prec) == P64) { typedef double S; __VA_ARGS__; }  \
        else if ((prec) == P32) { typedef float S; __VA_ARGS__; } \
        else { typedef bf16 S; __VA_ARGS__; }                  \
    } while (0)

int user_to_eo(wd_ctx *c, const void *user, bool user_double, int prec, void *even, void *odd, int nrhs) {
    if (nrhs <= 0) return WD_OK;
    const long n = (long)c->g.V * nrhs;
    const int th = 256;
    const unsigned blocks = (unsigned)((n + th - 1) / th);
    WD_DISPATCH_PREC(prec, S, {
        if (user_double) k_user_to_eo<double, S><<<blocks, th, 0, c->st>>>((const double *)user, even, odd, nrhs, c->g);
        else k_user_to_eo<float, S><<<blocks, th, 0, c->st>>>((const float *)user, even, odd, nrhs, c->g);
    });
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int eo_to_user(wd_ctx *c, const void *even, const void *odd, int prec, void *user, bool user_double, int nrhs) {
    if (nrhs <= 0) return WD_OK;
    const long n = (long)c->g.V * nrhs;
    const int th = 256;
    const unsigned blocks = (unsigned)((n + th - 1) / th);
    WD_DISPATCH_PREC(prec, S, {
        if (user_double) k_eo_to_user<S, double><<<blocks, th, 0, c->st>>>(even, odd, (double *)user, nrhs, c->g);
        else k_eo_to_user<S, float><<<blocks, th, 0, c->st>>>(even, odd, (float *)user, nrhs, c->g);
    });
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// ---- chunk-flat kernels ---------------------------------------------------
// When every operand of a kernel has the same precision, chunk q of one RHS
// holds the same complex components in each operand (in the eo layout and in
// the flat coarse layout alike), so the kernel can stream each RHS as one
// run of 16-byte chunks: no site arithmetic, UNR independent chunk loads per
// operand in flight per thread, grid (bpr, nrhs).  Used where it measured
// faster than the site kernels: the five-operand x, r update (6.0 against
// 4.8 TB/s) and the norms.
template <typename S> struct CIO;
template <> struct CIO<double> {
    static constexpr int NC = 1;
    __device__ __forceinline__ static void get(uint4 a, cx<double> v[1]) {
        v[0] = cmake(__hiloint2double(a.y, a.x), __hiloint2double(a.w, a.z));
    }
    __device__ __forceinline__ static uint4 put(const cx<double> v[1]) {
        return make_uint4(__double2loint(v[0].re), __double2hiint(v[0].re), __double2loint(v[0].im),
                          __double2hiint(v[0].im));
    }
};
template <> struct CIO<float> {
    static constexpr int NC = 2;
    __device__ __forceinline__ static void get(uint4 a, cx<float> v[2]) {
        v[0] = cmake(__uint_as_float(a.x), __uint_as_float(a.y));
        v[1] = cmake(__uint_as_float(a.z), __uint_as_float(a.w));
    }
    __device__ __forceinline__ static uint4 put(const cx<float> v[2]) {
        return make_uint4(__float_as_uint(v[0].re), __float_as_uint(v[0].im), __float_as_uint(v[1].re),
                          __float_as_uint(v[1].im));
    }
};
template <> struct CIO<bf16> {
    static constexpr int NC = 4;
    __device__ __forceinline__ static void get(uint4 a, cx<float> v[4]) {
        const unsigned w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            __nv_bfloat162 h;
            memcpy(&h, &w[j], 4);
            const float2 f = __bfloat1622float2(h);
            v[j] = cmake(f.x, f.y);
        }
    }
};

struct FlatRange { long q0, q1; };
__device__ __forceinline__ FlatRange flat_range(long nq) {
    const long chunk = (nq + gridDim.x - 1) / gridDim.x;
    FlatRange f;
    f.q0 = (long)blockIdx.x * chunk;
    f.q1 = f.q0 + chunk < nq ? f.q0 + chunk : nq;
    return f;
}

// x += alpha p + omega s; r = s - omega t; partials (rh, r) and |r|^2; all
// operands of one precision
template <typename S, int UNR>
__global__ void __launch_bounds__(256) k_xr_flat(void *x, void *r, const void *p, const void *s, const void *t,
                                                 const void *rh, const BiState *st, double *part, long nq,
                                                 int nrhs, int bpr) {
    pdl_wait();
    typedef typename RT_of<S>::type RT;
    constexpr int NC = CIO<S>::NC;
    if (!st[blockIdx.y].active) return;          // converged RHS: x, r stay as they are
    const size_t o = (size_t)blockIdx.y * nq;
    uint4 *X = (uint4 *)x + o, *Rr = (uint4 *)r + o;
    const uint4 *P = (const uint4 *)p + o, *Sv = (const uint4 *)s + o, *T = (const uint4 *)t + o,
                *RH = (const uint4 *)rh + o;
    const double2 a = st[blockIdx.y].alpha, w = st[blockIdx.y].omega;
    const cx<RT> al = cmake((RT)a.x, (RT)a.y), om = cmake((RT)w.x, (RT)w.y), mom = cmake(-om.re, -om.im);
    const FlatRange F = flat_range(nq);
    cx<RT> dot = cmake(RT(0), RT(0));
    RT nn = 0;
    for (long q = F.q0 + threadIdx.x; q < F.q1; q += UNR * blockDim.x) {
        uint4 ux[UNR], up[UNR], us[UNR], ut[UNR], uh[UNR];
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const long qq = q + k * (long)blockDim.x;
            const bool in = qq < F.q1;
            const uint4 z = make_uint4(0, 0, 0, 0);
            ux[k] = in ? X[qq] : z;
            up[k] = in ? __ldg(P + qq) : z;
            us[k] = in ? __ldg(Sv + qq) : z;
            ut[k] = in ? __ldg(T + qq) : z;
            uh[k] = in ? __ldg(RH + qq) : z;
        }
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            cx<RT> xv[NC], pv[NC], sv[NC], tv[NC], hv[NC];
            CIO<S>::get(ux[k], xv);
            CIO<S>::get(up[k], pv);
            CIO<S>::get(us[k], sv);
            CIO<S>::get(ut[k], tv);
            CIO<S>::get(uh[k], hv);
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                cfma(xv[j], al, pv[j]);
                cfma(xv[j], om, sv[j]);
                cx<RT> rn = sv[j];
                cfma(rn, mom, tv[j]);
                cfma_conj(dot, hv[j], rn);
                nn += rn.re * rn.re + rn.im * rn.im;
                tv[j] = rn;
            }
            const long qq = q + k * (long)blockDim.x;
            if (qq < F.q1) {
                X[qq] = CIO<S>::put(xv);
                Rr[qq] = CIO<S>::put(tv);
            }
        }
    }
    double d[3] = {(double)dot.re, (double)dot.im, (double)nn};
    block_partials<3>(d, part, nrhs, bpr);
}

// partial |a|^2 over nq chunks per RHS
template <typename S, int UNR>
__global__ void __launch_bounds__(256) k_norm2_flat(const void *a, double *part, long nq, int nrhs, int bpr) {
    typedef typename RT_of<S>::type RT;
    constexpr int NC = CIO<S>::NC;
    const uint4 *A = (const uint4 *)a + (size_t)blockIdx.y * nq;
    const FlatRange F = flat_range(nq);
    RT acc = 0;
    for (long q = F.q0 + threadIdx.x; q < F.q1; q += UNR * blockDim.x) {
        uint4 ua[UNR];
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const long qq = q + k * (long)blockDim.x;
            ua[k] = qq < F.q1 ? __ldg(A + qq) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            cx<RT> v[NC];
            CIO<S>::get(ua[k], v);
#pragma unroll
            for (int j = 0; j < NC; ++j) acc += v[j].re * v[j].re + v[j].im * v[j].im;
        }
    }
    double d[1] = {(double)acc};
    block_partials<1>(d, part, nrhs, bpr);
}

// |a|^2 of FP64 fields on the FP32 pipes (FP64 arithmetic runs at a small
// fraction of the FP32 rate on this GPU).  Each double v = m 2^e, m in [1, 2),
// is split by integer operations into mh (the leading 24 significand bits)
// and ml (the remaining 29 bits, as a float, to 2^-24 of themselves), so
// v = (mh + ml) 2^e to about 2^-47 relative.  A thread keeps one running
// exponent E (the largest e seen) and an unevaluated float pair (S, C) with
// sum v^2 = (S + C) 2^(2E): each term (mh + ml)^2 2^(2(e - E)) enters as an
// exact product mh^2 (rounded product plus its FMA remainder) plus 2 mh ml,
// added to S by TwoSum (Knuth); when E grows, S and C are rescaled by a
// power of two.  Terms more than 2^126 below the running maximum are dropped
// (they lie far below the pair's precision).  Relative accuracy ~1e-13;
// subnormal inputs count as zero; an infinity or NaN makes the result NaN.
struct Split64 {
    float mh, ml;
    int e;
};
__device__ __forceinline__ Split64 split64(unsigned lo, unsigned hi, bool &nf) {
    Split64 r;
    const int ef = (int)((hi >> 20) & 0x7FFu);
    if (ef == 0 || ef == 0x7FF) {
        nf |= ef == 0x7FF;
        r.mh = r.ml = 0.f;
        r.e = -4096;
        return r;
    }
    r.e = ef - 1023;
    r.mh = __int_as_float(0x3F800000 | (int)((hi & 0xFFFFFu) << 3) | (int)(lo >> 29));
    r.ml = __fmul_rn(__uint2float_rn(lo & 0x1FFFFFFFu), 0x1p-52f);
    return r;
}
// 2^d as a float for d <= 0; 0 below the normal range
__device__ __forceinline__ float pow2f_le0(int d) { return d >= -126 ? __int_as_float((127 + d) << 23) : 0.f; }

template <int UNR>
__global__ void __launch_bounds__(256) k_norm2_f64(const void *a, double *part, long nq, int nrhs, int bpr) {
    const uint4 *A = (const uint4 *)a + (size_t)blockIdx.y * nq;
    const FlatRange F = flat_range(nq);
    float S = 0.f, C = 0.f;
    int E = -4096;
    bool nf = false;
    for (long q = F.q0 + threadIdx.x; q < F.q1; q += UNR * blockDim.x) {
        uint4 ua[UNR];
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const long qq = q + k * (long)blockDim.x;
            ua[k] = qq < F.q1 ? __ldg(A + qq) : make_uint4(0, 0, 0, 0);
        }
        Split64 v[2 * UNR];
        int Eg = -4096;
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            v[2 * k] = split64(ua[k].x, ua[k].y, nf);
            v[2 * k + 1] = split64(ua[k].z, ua[k].w, nf);
            Eg = max(Eg, max(v[2 * k].e, v[2 * k + 1].e));
        }
        if (Eg > E) {
            const float sc = E == -4096 ? 0.f : pow2f_le0(2 * (E - Eg));
            S = __fmul_rn(S, sc);
            C = __fmul_rn(C, sc);
            E = Eg;
        }
#pragma unroll
        for (int j = 0; j < 2 * UNR; ++j) {
            const float sc = v[j].e == -4096 ? 0.f : pow2f_le0(v[j].e - E);
            const float h = __fmul_rn(v[j].mh, sc), l = __fmul_rn(v[j].ml, sc);
            const float p = __fmul_rn(h, h);
            const float err = __fadd_rn(__fmaf_rn(h, h, -p), __fmul_rn(__fmul_rn(2.f, h), l));
            const float s1 = __fadd_rn(S, p), bb = __fsub_rn(s1, S);
            const float e1 = __fadd_rn(__fsub_rn(S, __fsub_rn(s1, bb)), __fsub_rn(p, bb));
            S = s1;
            C = __fadd_rn(C, __fadd_rn(e1, err));
        }
    }
    double acc = 0.0;
    if (E != -4096) {
        const double t = __hiloint2double((E + 1023) << 20, 0);     // 2^E, E in [-1022, 1023]
        acc = (((double)S + (double)C) * t) * t;
    }
    if (nf) acc = __longlong_as_double(0x7FF8000000000000LL);
    double d[1] = {acc};
    block_partials<1>(d, part, nrhs, bpr);
}

// |a|^2 of double-float fields (each complex a float4 (re.h, im.h, re.l,
// im.l), value h + l) with the same running-exponent float-pair sum as
// k_norm2_f64.  The pair is first renormalised by TwoSum (a stencil output
// need not be: after cancellation h can be 0 with l not), then v = (mh + ml)
// 2^e with e the exponent of h, mh its significand and ml = l 2^-e carried
// with the sign of l relative to h.
__device__ __forceinline__ Split64 split_ddl(float h0, float l0, bool &nf) {
    const float h = __fadd_rn(h0, l0), bb = __fsub_rn(h, h0);
    const float l = __fadd_rn(__fsub_rn(h0, __fsub_rn(h, bb)), __fsub_rn(l0, bb));
    Split64 r;
    const unsigned hb = __float_as_uint(h);
    const int ef = (int)((hb >> 23) & 0xFFu);
    if (ef == 0 || ef == 0xFF) {
        nf |= ef == 0xFF;
        r.mh = r.ml = 0.f;
        r.e = -4096;
        return r;
    }
    r.e = ef - 127;
    r.mh = __int_as_float(0x3F800000 | (int)(hb & 0x7FFFFFu));
    r.ml = ldexpf((hb >> 31) ? -l : l, -r.e);
    return r;
}

template <int UNR>
__global__ void __launch_bounds__(256) k_norm2_ddl(const void *a, double *part, long nq, int nrhs, int bpr) {
    const float4 *A = (const float4 *)a + (size_t)blockIdx.y * nq;
    const FlatRange F = flat_range(nq);
    float S = 0.f, C = 0.f;
    int E = -4096;
    bool nf = false;
    for (long q = F.q0 + threadIdx.x; q < F.q1; q += UNR * blockDim.x) {
        float4 ua[UNR];
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            const long qq = q + k * (long)blockDim.x;
            ua[k] = qq < F.q1 ? __ldg(A + qq) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        Split64 v[2 * UNR];
        int Eg = -4096;
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
            v[2 * k] = split_ddl(ua[k].x, ua[k].z, nf);
            v[2 * k + 1] = split_ddl(ua[k].y, ua[k].w, nf);
            Eg = max(Eg, max(v[2 * k].e, v[2 * k + 1].e));
        }
        if (Eg > E) {
            const float sc = E == -4096 ? 0.f : pow2f_le0(2 * (E - Eg));
            S = __fmul_rn(S, sc);
            C = __fmul_rn(C, sc);
            E = Eg;
        }
#pragma unroll
        for (int j = 0; j < 2 * UNR; ++j) {
            const float sc = v[j].e == -4096 ? 0.f : pow2f_le0(v[j].e - E);
            const float h = __fmul_rn(v[j].mh, sc), l = __fmul_rn(v[j].ml, sc);
            const float p = __fmul_rn(h, h);
            const float err = __fadd_rn(__fmaf_rn(h, h, -p), __fmul_rn(__fmul_rn(2.f, h), l));
            const float s1 = __fadd_rn(S, p), bb = __fsub_rn(s1, S);
            const float e1 = __fadd_rn(__fsub_rn(S, __fsub_rn(s1, bb)), __fsub_rn(p, bb));
            S = s1;
            C = __fadd_rn(C, __fadd_rn(e1, err));
        }
    }
    double acc = 0.0;
    if (E != -4096) {
        const double t = __hiloint2double((E + 1023) << 20, 0);     // 2^E
        acc = (((double)S + (double)C) * t) * t;
    }
    if (nf) acc = __longlong_as_double(0x7FF8000000000000LL);
    double d[1] = {acc};
    block_partials<1>(d, part, nrhs, bpr);
}

// FP32 copy of a double-float field times a per-RHS FP64 scale, on the FP32
// pipes: out = RN(h + l) ms 2^es with scale = ms 2^es (ms rounded to FP32),
// the power of two applied by ldexpf, so the scale may lie outside the FP32
// range as long as the product does not.  Item i of a RHS is (site s, FP32
// chunk j): the double-float chunks 2j, 2j+1 of s in, FP32 chunk j out.
template <bool FL>
__global__ void __launch_bounds__(256) k_ddl_to_f32(const void *a, void *b, const double *scale, long units) {
    const long per = 6 * units;
    const float4 *A = (const float4 *)a + (size_t)blockIdx.y * 12 * units;
    float4 *B = (float4 *)b + (size_t)blockIdx.y * per;
    float ms = 1.f;
    int es = 0;
    if (scale) {
        const double sd = scale[blockIdx.y];
        bool nf = false;
        const Split64 sp = split64(__double2loint(sd), __double2hiint(sd), nf);
        if (sp.e == -4096) { ms = nf ? __int_as_float(0x7FC00000) : 0.f; }
        else {
            ms = __fadd_rn(sp.mh, sp.ml);
            es = sp.e;
            if (sd < 0) ms = -ms;
        }
    }
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < per; i += (long)gridDim.x * blockDim.x) {
        long i0, i1, o;
        if (FL) {
            const long u = i / 6, j = i - 6 * u;
            i0 = 12 * u + 2 * j; i1 = i0 + 1; o = i;
        } else {
            const long j = i / units, s = i - j * units;
            i0 = 2 * j * units + s; i1 = i0 + units; o = i;
        }
        const float4 v0 = __ldg(A + i0), v1 = __ldg(A + i1);
        float4 r;
        r.x = ldexpf(__fmul_rn(__fadd_rn(v0.x, v0.z), ms), es);
        r.y = ldexpf(__fmul_rn(__fadd_rn(v0.y, v0.w), ms), es);
        r.z = ldexpf(__fmul_rn(__fadd_rn(v1.x, v1.z), ms), es);
        r.w = ldexpf(__fmul_rn(__fadd_rn(v1.y, v1.w), ms), es);
        B[o] = r;
    }
}

// x (double-float layout) += scale * e (FP32 field) in double-float
// arithmetic, item (site, FP32 chunk j) as in k_ddl_to_f32.  The scale
// (FP64, per RHS) is split into sh + sl (sh: its leading 24 bits, sl the
// next 24, each as a float scaled by ldexpf); the product (sh + sl) e keeps
// the exact FMA error of sh e; the sum with x uses TwoSum twice and ends
// renormalised (|l| <= ulp(h) / 2).
__device__ __forceinline__ void dd_axpy_one(float &xh, float &xl, float sh, float sl, float e) {
    const float p = __fmul_rn(sh, e);
    const float q = __fmaf_rn(sl, e, __fmaf_rn(sh, e, -p));         // error of p plus sl e
    const float s = __fadd_rn(xh, p), bb = __fsub_rn(s, xh);
    const float err = __fadd_rn(__fsub_rn(xh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    const float t = __fadd_rn(xl, __fadd_rn(q, err));
    xh = __fadd_rn(s, t);                                            // TwoSum: xl the exact error of xh
    const float b2 = __fsub_rn(xh, s);
    xl = __fadd_rn(__fsub_rn(s, __fsub_rn(xh, b2)), __fsub_rn(t, b2));
}

template <bool FL>
__global__ void __launch_bounds__(256) k_axpy_ddl(void *x, const void *e, const double *scale, long units) {
    const long per = 6 * units;
    float4 *X = (float4 *)x + (size_t)blockIdx.y * 12 * units;
    const float4 *Ev = (const float4 *)e + (size_t)blockIdx.y * per;
    const double sd = scale[blockIdx.y];
    bool nf = false;
    const Split64 sp = split64(__double2loint(sd), __double2hiint(sd), nf);
    if (sp.e == -4096) return;                  // zero scale: a converged RHS, x unchanged
    const float sg = sd < 0 ? -1.f : 1.f;
    const float sh = ldexpf(sg * sp.mh, sp.e), sl = ldexpf(sg * sp.ml, sp.e);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < per; i += (long)gridDim.x * blockDim.x) {
        long i0, i1;
        if (FL) {
            const long u = i / 6, j = i - 6 * u;
            i0 = 12 * u + 2 * j; i1 = i0 + 1;
        } else {
            const long j = i / units, st = i - j * units;
            i0 = 2 * j * units + st; i1 = i0 + units;
        }
        const float4 ev = __ldg(Ev + i);
        float4 a = X[i0], b = X[i1];
        dd_axpy_one(a.x, a.z, sh, sl, ev.x);
        dd_axpy_one(a.y, a.w, sh, sl, ev.y);
        dd_axpy_one(b.x, b.z, sh, sl, ev.z);
        dd_axpy_one(b.y, b.w, sh, sl, ev.w);
        X[i0] = a;
        X[i1] = b;
    }
}

// h + l (a renormalised double-float pair) as a double, assembled with
// integer operations: h's significand widened to 53 bits, l added in units
// of its last bit (truncating what falls below), one renormalising shift.
// Within one FP64 ulp of h + l.  h zero, subnormal or not finite: FP64 adds.
__device__ __forceinline__ double ddpair_to_double(float h, float l) {
    const unsigned hb = __float_as_uint(h), lb = __float_as_uint(l);
    const int eh = (int)((hb >> 23) & 0xFFu), el = (int)((lb >> 23) & 0xFFu);
    if (eh == 0 || eh == 0xFF) return __dadd_rn((double)h, (double)l);
    unsigned long long M = (1ull << 52) | ((unsigned long long)(hb & 0x7FFFFFu) << 29);
    int E = eh - 127;                                            // h + l = M 2^(E - 52)
    if (el != 0) {
        const unsigned long long Ml = (1ull << 23) | (lb & 0x7FFFFFu);
        const int sh = (el - 150) - (E - 52);                    // <= 5 for a renormalised pair
        const unsigned long long add = sh >= 0 ? (sh <= 28 ? Ml << sh : 0ull) : (sh > -64 ? Ml >> -sh : 0ull);
        if ((hb ^ lb) >> 31) M -= add;
        else M += add;
        if (M >> 53) { M >>= 1; E += 1; }
        else if (!(M >> 52)) { M <<= 1; E -= 1; }
    }
    const unsigned long long bits = ((unsigned long long)(hb >> 31) << 63) |
                                    ((unsigned long long)(E + 1023) << 52) | (M & ((1ull << 52) - 1));
    return __longlong_as_double((long long)bits);
}

__global__ void __launch_bounds__(256) k_ddl_to_f64(const float4 *a, double2 *b, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float4 v = __ldg(a + i);
        b[i] = make_double2(ddpair_to_double(v.x, v.z), ddpair_to_double(v.y, v.w));
    }
}

// ---- conversions and mixed axpy ---------------------------------------------
template <typename SA, typename SB, bool FL>
__global__ void k_convert(const void *a, void *b, const double *scale, long Vh, long n) {
    typedef typename RT_of<SA>::type RA;
    for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < n; u += (long)gridDim.x * blockDim.x) {
        cx<RA> v[12];
        ldsite<SA, RA, FL>(a, Vh, u, v);
        if (scale) {
            const RA s = (RA)scale[u / Vh];
#pragma unroll
            for (int j = 0; j < 12; ++j) v[j] = s * v[j];
        }
        stsite<SB, RA, FL>(b, Vh, u, v);
    }
}

template <typename SE, bool FL>
__global__ void k_axpy_mixed(double *x, const void *e, const double *scale, long Vh, long n) {
    for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < n; u += (long)gridDim.x * blockDim.x) {
        const double s = scale[u / Vh];
        cx<double> xv[12], ev[12];
        ldsite<double, double, FL>(x, Vh, u, xv);
        ldsite<SE, double, FL>(e, Vh, u, ev);
#pragma unroll
        for (int j = 0; j < 12; ++j) { xv[j].re += s * ev[j].re; xv[j].im += s * ev[j].im; }
        stsite<double, double, FL>(x, Vh, u, xv);
    }
}

static unsigned ew_blocks(long n) {
    long b = (n + 255) / 256;
    long cap = 148L * 16;
    return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

#define WD_DISPATCH_FLAT(flat, FL, ...)                 \
    do {                                                \
        if (flat) { constexpr bool FL = true; __VA_ARGS__; } \
        else { constexpr bool FL = false; __VA_ARGS__; }     \
    } while (0)

int blas_copy_convert(wd_ctx *c, const Space &sp, int ps, const void *src, int pd, void *dst, int nrhs,
                      const double *scale) {
    const long Vh = sp.units, n = Vh * nrhs;
    if (n == 0) return WD_OK;
    if (ps == PDDL) {
        if (pd != P32) { set_error("copy: double-float source needs an FP32 destination"); return WD_EINVAL; }
        const unsigned bx = (unsigned)std::max(1, std::min(64, reduction_bpr(Vh, nrhs)));
        if (sp.flat) k_ddl_to_f32<true><<<dim3(bx, nrhs), 256, 0, c->st>>>(src, dst, scale, Vh);
        else k_ddl_to_f32<false><<<dim3(bx, nrhs), 256, 0, c->st>>>(src, dst, scale, Vh);
        c->launches++;
        WD_CUDA(cudaGetLastError());
        return WD_OK;
    }
    WD_DISPATCH_FLAT(sp.flat, FL, WD_DISPATCH_PREC(ps, SA, WD_DISPATCH_PREC(pd, SB,
        k_convert<SA, SB, FL><<<ew_blocks(n), 256, 0, c->st>>>(src, dst, scale, Vh, n))));
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int blas_axpy_ddl(wd_ctx *c, const Space &sp, void *x, const void *e, const double *scale, int nrhs) {
    if (nrhs <= 0 || sp.units == 0) return WD_OK;
    const unsigned bx = (unsigned)std::max(1, std::min(64, reduction_bpr(sp.units, nrhs)));
    if (sp.flat) k_axpy_ddl<true><<<dim3(bx, nrhs), 256, 0, c->st>>>(x, e, scale, sp.units);
    else k_axpy_ddl<false><<<dim3(bx, nrhs), 256, 0, c->st>>>(x, e, scale, sp.units);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int blas_ddl_to_f64(wd_ctx *c, const Space &sp, const void *x, double *x64, int nrhs) {
    const long n = 12L * sp.units * nrhs;
    if (n == 0) return WD_OK;
    k_ddl_to_f64<<<ew_blocks(n / 12), 256, 0, c->st>>>((const float4 *)x, (double2 *)x64, n);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int blas_axpy_mixed(wd_ctx *c, const Space &sp, double *x, int pe, const void *e, const double *scale, int nrhs) {
    const long Vh = sp.units, n = Vh * nrhs;
    if (n == 0) return WD_OK;
    WD_DISPATCH_FLAT(sp.flat, FL, WD_DISPATCH_PREC(pe, SE,
        k_axpy_mixed<SE, FL><<<ew_blocks(n), 256, 0, c->st>>>(x, e, scale, Vh, n)));
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int blas_zero(wd_ctx *c, void *p, size_t bytes) {
    WD_CUDA(cudaMemsetAsync(p, 0, bytes, c->st));
    return WD_OK;
}

// ---- norms -------------------------------------------------------------------
__global__ void k_sum_partials(const double *part, double *out, int nrhs, int bpr) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrhs; r += gridDim.x * blockDim.x)
        out[r] = sum_part(part, 0, r, nrhs, bpr);
}

int blas_norm2(wd_ctx *c, const Space &sp, int prec, const void *a, int nrhs, double *out) {
    if (nrhs <= 0) return WD_OK;
    const int bpr = reduction_bpr(sp.units, nrhs);
    double *part;
    WD_TRY(ws_get(c, "norm_part", sizeof(double) * bpr * nrhs, (void **)&part));
    dim3 grid(bpr, nrhs);
    if (prec == P64)
        k_norm2_f64<4><<<grid, 256, 0, c->st>>>(a, part, 12L * sp.units, nrhs, bpr);
    else if (prec == PDDL)
        k_norm2_ddl<4><<<grid, 256, 0, c->st>>>(a, part, 12L * sp.units, nrhs, bpr);
    else if (prec == P32)
        k_norm2_flat<float, 4><<<grid, 256, 0, c->st>>>(a, part, 6L * sp.units, nrhs, bpr);
    else
        k_norm2_flat<bf16, 4><<<grid, 256, 0, c->st>>>(a, part, 3L * sp.units, nrhs, bpr);
    k_sum_partials<<<(nrhs + 127) / 128, 128, 0, c->st>>>(part, out, nrhs, bpr);
    c->launches += 2;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// ---- BiCGStab ------------------------------------------------------------------
// init: x = 0, r = rh = b, p = b (operator precision); partial |b|^2
template <typename SW, typename SP, bool FL>
__global__ void k_bicg_init(const void *b, void *x, void *r, void *rh, void *p, double *part, long Vh, int nrhs,
                            int bpr) {
    typedef typename RT_of<SW>::type RT;
    Range R = my_range(Vh);
    RT acc = 0;
    for (long u = R.g0 + threadIdx.x; u < R.g1; u += blockDim.x) {
        cx<RT> v[12], z[12];
        ldsite<SW, RT, FL>(b, Vh, u, v);
#pragma unroll
        for (int j = 0; j < 12; ++j) { z[j] = cmake(RT(0), RT(0)); acc += v[j].re * v[j].re + v[j].im * v[j].im; }
        stsite<SW, RT, FL>(x, Vh, u, z);
        stsite<SW, RT, FL>(r, Vh, u, v);
        stsite<SW, RT, FL>(rh, Vh, u, v);
        stsite<SP, RT, FL>(p, Vh, u, v);
    }
    double d[1] = {(double)acc};
    block_partials<1>(d, part, nrhs, bpr);
}

// The iteration kernels below skip every RHS whose state is inactive
// (converged or broken down): its x and r keep their final values, and the
// other fields of that RHS are neither read nor written again in this run.
// Stencil launches inside the run walk the list of the active RHS that
// k_scal_init / k_scal_beta build after every update of the states
// (HopArgs::alist).

// list[0 .. count) = the active RHS in ascending order (count: the number
// k_scal_init / k_scal_beta store); run by the whole single block of those
// kernels after their state updates, fixed order
__device__ void build_active_list(const BiState *st, int nrhs, int *list) {
    __shared__ int wc[32];
    __shared__ int base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nrhs; c0 += blockDim.x) {
        const int r = c0 + threadIdx.x;
        const bool a = r < nrhs && st[r].active;
        const unsigned m = __ballot_sync(0xffffffffu, a);
        if (lane == 0) wc[wid] = __popc(m);
        __syncthreads();
        int off = base;
        for (int w = 0; w < wid; ++w) off += wc[w];
        if (a) list[off + __popc(m & ((1u << lane) - 1u))] = r;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < nw; ++w) tot += wc[w];
            base += tot;
        }
        __syncthreads();
    }
}

__global__ void k_scal_init(BiState *st, const double *part, const double *bnorm2, double tol2, int nrhs, int bpr,
                            int *count, int *list) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
        const double rr = sum_part(part, 0, r, nrhs, bpr);
        BiState s;
        s.rho = make_double2(rr, 0.0);
        s.alpha = make_double2(0.0, 0.0);
        s.omega = make_double2(0.0, 0.0);
        s.beta = make_double2(0.0, 0.0);
        s.rr = rr;
        s.bb = bnorm2 ? bnorm2[r] : rr;
        s.thr = tol2 * s.bb;
        s.iters = 0;
        s.flag = 0;
        s.pad = 0;
        s.active = (rr > s.thr && rr > 0.0 && isfinite(rr)) ? 1 : 0;
        if (!isfinite(rr)) s.flag = 1;
        st[r] = s;
        if (s.active) atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *count = cnt;
    build_active_list(st, nrhs, list);
}

// partial sums of conj(a).b (slots 0, 1) and optionally |a|^2 (slot 2)
template <typename SA, typename SB, bool NORMA, bool FL>
__global__ void k_dot_part(const void *a, const void *b, double *part, long Vh, int nrhs, int bpr,
                           const BiState *st) {
    pdl_wait();
    typedef typename RT_of<SA>::type RT;
    if (st && !st[blockIdx.y].active) return;    // converged RHS: partials unused
    Range R = my_range(Vh);
    cx<RT> acc = cmake(RT(0), RT(0));
    RT nn = 0;
    for (long u = R.g0 + threadIdx.x; u < R.g1; u += blockDim.x) {
        cx<RT> va[12], vb[12];
        ldsite<SA, RT, FL>(a, Vh, u, va);
        ldsite<SB, RT, FL>(b, Vh, u, vb);
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            cfma_conj(acc, va[j], vb[j]);
            if (NORMA) nn += va[j].re * va[j].re + va[j].im * va[j].im;
        }
    }
    if (NORMA) {
        double d[3] = {(double)acc.re, (double)acc.im, (double)nn};
        block_partials<3>(d, part, nrhs, bpr);
    } else {
        double d[2] = {(double)acc.re, (double)acc.im};
        block_partials<2>(d, part, nrhs, bpr);
    }
}

__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double den = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ bool zfinite(double2 a) { return isfinite(a.x) && isfinite(a.y); }

// alpha = rho / (r_hat, v) of one active RHS; breakdown masks the RHS
__device__ void scal_alpha(BiState &s, double2 d) {
    const double2 al = zdiv(s.rho, d);
    if ((d.x == 0.0 && d.y == 0.0) || !zfinite(al)) {
        s.active = 0; s.flag = 1;
        s.alpha = make_double2(0, 0); s.omega = make_double2(0, 0); s.beta = make_double2(0, 0);
        return;
    }
    s.alpha = al;
}

// omega = (t, s) / |t|^2 of one active RHS
__device__ void scal_omega(BiState &s, double2 ts, double tt) {
    if (tt == 0.0) { s.omega = make_double2(0, 0); return; }   // t = A s = 0 => s = 0
    const double2 om = make_double2(ts.x / tt, ts.y / tt);
    if (!zfinite(om)) { s.active = 0; s.flag = 1; s.omega = make_double2(0, 0); s.alpha = make_double2(0, 0); return; }
    s.omega = om;
}

__global__ void k_scal_alpha(BiState *st, const double *part, int nrhs, int bpr) {
    pdl_wait();
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrhs; r += gridDim.x * blockDim.x) {
        BiState &s = st[r];
        if (!s.active) { s.alpha = make_double2(0, 0); continue; }
        scal_alpha(s, make_double2(sum_part(part, 0, r, nrhs, bpr), sum_part(part, 1, r, nrhs, bpr)));
    }
}

__global__ void k_scal_omega(BiState *st, const double *part, int nrhs, int bpr) {
    pdl_wait();
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrhs; r += gridDim.x * blockDim.x) {
        BiState &s = st[r];
        if (!s.active) { s.omega = make_double2(0, 0); continue; }
        scal_omega(s, make_double2(sum_part(part, 0, r, nrhs, bpr), sum_part(part, 1, r, nrhs, bpr)),
                   sum_part(part, 2, r, nrhs, bpr));
    }
}

__global__ void k_scal_beta(BiState *st, const double *part, int nrhs, int bpr, int *count, int *list) {
    pdl_wait();
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
        BiState &s = st[r];
        if (!s.active) { s.beta = make_double2(0, 0); continue; }
        const double2 rho = make_double2(sum_part(part, 0, r, nrhs, bpr), sum_part(part, 1, r, nrhs, bpr));
        const double rr = sum_part(part, 2, r, nrhs, bpr);
        s.iters++;
        s.rr = rr;
        if (!isfinite(rr)) { s.active = 0; s.flag = 1; }
        else if (rr <= s.thr) { s.active = 0; }
        else if ((s.omega.x == 0.0 && s.omega.y == 0.0) || (s.rho.x == 0.0 && s.rho.y == 0.0)) { s.active = 0; s.flag = 1; }
        if (!s.active) {
            s.alpha = make_double2(0, 0); s.omega = make_double2(0, 0); s.beta = make_double2(0, 0);
            continue;
        }
        s.beta = zmul(zdiv(rho, s.rho), zdiv(s.alpha, s.omega));
        s.rho = rho;
        atomicAdd(&cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *count = cnt;
    build_active_list(st, nrhs, list);
}

// s = r - alpha v
template <typename SW, typename SP, bool FL>
__global__ void k_bicg_s(const void *r, const void *v, void *s, const BiState *st, long Vh, long n) {
    pdl_wait();
    typedef typename RT_of<SW>::type RT;
    for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < n; u += (long)gridDim.x * blockDim.x) {
        if (!st[u / Vh].active) continue;
        const double2 a = st[u / Vh].alpha;
        const cx<RT> mal = cmake((RT)-a.x, (RT)-a.y);
        cx<RT> rv[12], vv[12];
        ldsite<SW, RT, FL>(r, Vh, u, rv);
        ldsite<SW, RT, FL>(v, Vh, u, vv);
#pragma unroll
        for (int j = 0; j < 12; ++j) cfma(rv[j], mal, vv[j]);
        stsite<SP, RT, FL>(s, Vh, u, rv);
    }
}

// x += alpha p + omega s; r = s - omega t; partials (rh, r) and |r|^2
template <typename SW, typename SP, bool FL>
__global__ void k_bicg_xr(void *x, void *r, const void *p, const void *s, const void *t, const void *rh,
                          const BiState *st, double *part, long Vh, int nrhs, int bpr) {
    pdl_wait();
    typedef typename RT_of<SW>::type RT;
    if (!st[blockIdx.y].active) return;          // converged RHS: x, r stay as they are
    Range R = my_range(Vh);
    const double2 a = st[blockIdx.y].alpha, w = st[blockIdx.y].omega;
    const cx<RT> al = cmake((RT)a.x, (RT)a.y), om = cmake((RT)w.x, (RT)w.y), mom = cmake(-om.re, -om.im);
    cx<RT> dot = cmake(RT(0), RT(0));
    RT nn = 0;
    for (long u = R.g0 + threadIdx.x; u < R.g1; u += blockDim.x) {
        cx<RT> xv[12], pv[12], sv[12], tv[12];
        ldsite<SW, RT, FL>(x, Vh, u, xv);
        ldsite<SP, RT, FL>(p, Vh, u, pv);
        ldsite<SP, RT, FL>(s, Vh, u, sv);
#pragma unroll
        for (int j = 0; j < 12; ++j) { cfma(xv[j], al, pv[j]); cfma(xv[j], om, sv[j]); }
        stsite<SW, RT, FL>(x, Vh, u, xv);
        ldsite<SW, RT, FL>(t, Vh, u, tv);
        ldsite<SW, RT, FL>(rh, Vh, u, pv);
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            cx<RT> rn = sv[j];
            cfma(rn, mom, tv[j]);
            cfma_conj(dot, pv[j], rn);
            nn += rn.re * rn.re + rn.im * rn.im;
            tv[j] = rn;
        }
        stsite<SW, RT, FL>(r, Vh, u, tv);
    }
    double d[3] = {(double)dot.re, (double)dot.im, (double)nn};
    block_partials<3>(d, part, nrhs, bpr);
}

// p = r + beta (p - omega v)
template <typename SW, typename SP, bool FL>
__global__ void k_bicg_p(const void *r, void *p, const void *v, const BiState *st, long Vh, long n) {
    pdl_wait();
    typedef typename RT_of<SW>::type RT;
    for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < n; u += (long)gridDim.x * blockDim.x) {
        const BiState &S = st[u / Vh];
        if (!S.active) continue;
        const cx<RT> be = cmake((RT)S.beta.x, (RT)S.beta.y), mom = cmake((RT)-S.omega.x, (RT)-S.omega.y);
        cx<RT> rv[12], pv[12], vv[12];
        ldsite<SW, RT, FL>(r, Vh, u, rv);
        ldsite<SP, RT, FL>(p, Vh, u, pv);
        ldsite<SW, RT, FL>(v, Vh, u, vv);
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            cfma(pv[j], mom, vv[j]);
            cfma(rv[j], be, pv[j]);
        }
        stsite<SP, RT, FL>(p, Vh, u, rv);
    }
}

#define WD_DISPATCH_PAIR(pw, pp, SW, SP, ...)                                         \
    do {                                                                              \
        if ((pw) == P64) { typedef double SW; typedef double SP; __VA_ARGS__; }       \
        else if ((pp) == P32) { typedef float SW; typedef float SP; __VA_ARGS__; }    \
        else { typedef float SW; typedef bf16 SP; __VA_ARGS__; }                      \
    } while (0)

int bicg_init(wd_ctx *c, int pw, int pp, BiVecs &V, const void *b, int nrhs, double tol_rel,
              const double *bnorm2_dev) {
    const long Vh = V.sp.units;
    dim3 grid(V.bpr, nrhs);
    WD_DISPATCH_FLAT(V.sp.flat, FL, WD_DISPATCH_PAIR(pw, pp, SW, SP,
        k_bicg_init<SW, SP, FL><<<grid, 256, 0, c->st>>>(b, V.x, V.r, V.rh, V.p, V.part, Vh, nrhs, V.bpr)));
    k_scal_init<<<1, 256, 0, c->st>>>(V.st, V.part, bnorm2_dev, tol_rel * tol_rel, nrhs, V.bpr, V.count, V.alist);
    c->launches += 2;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// BLAS half after v = A p: alpha = rho / (rh, v), s = r - alpha v
int bicg_after_v(wd_ctx *c, int pw, int pp, BiVecs &V, int nrhs) {
    const long Vh = V.sp.units, n = Vh * nrhs;
    dim3 grid(V.bpr, nrhs);
    const unsigned eb = ew_blocks(n);
    WD_DISPATCH_FLAT(V.sp.flat, FL, WD_DISPATCH_PAIR(pw, pp, SW, SP, {
        launch_pdl(k_dot_part<SW, SW, false, FL>, grid, dim3(256), 0, c->st, (const void *)V.rh, (const void *)V.v,
                   V.part, Vh, nrhs, V.bpr, (const BiState *)V.st);
        launch_pdl(k_scal_alpha, dim3((nrhs + 127) / 128), dim3(128), 0, c->st, V.st, (const double *)V.part, nrhs,
                   V.bpr);
        launch_pdl(k_bicg_s<SW, SP, FL>, dim3(eb), dim3(256), 0, c->st, (const void *)V.r, (const void *)V.v, V.s,
                   (const BiState *)V.st, Vh, n);
    }));
    c->launches += 3;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// the x and r update of one RHS precision pair: chunk-flat when the search
// direction has the iterate's precision, per site (with conversions) when it
// is BF16
template <typename SW, typename SP, bool FL> struct XrUpdate {
    static void run(wd_ctx *c, BiVecs &V, int nrhs) {
        k_bicg_xr<SW, SP, FL><<<dim3(V.bpr, nrhs), 256, 0, c->st>>>(V.x, V.r, V.p, V.s, V.t, V.rh, V.st, V.part,
                                                                    V.sp.units, nrhs, V.bpr);
    }
};
template <typename S, bool FL> struct XrUpdate<S, S, FL> {
    static void run(wd_ctx *c, BiVecs &V, int nrhs) {
        launch_pdl(k_xr_flat<S, 2>, dim3(V.bpr, nrhs), dim3(256), 0, c->st, V.x, V.r, (const void *)V.p,
                   (const void *)V.s, (const void *)V.t, (const void *)V.rh, (const BiState *)V.st, V.part,
                   (long)SIO<S>::NCH * V.sp.units, nrhs, V.bpr);
    }
};

// BLAS half after t = A s: omega, x and r updates, rho and beta, p update
int bicg_after_t(wd_ctx *c, int pw, int pp, BiVecs &V, int nrhs) {
    const long Vh = V.sp.units, n = Vh * nrhs;
    dim3 grid(V.bpr, nrhs);
    const unsigned eb = ew_blocks(n);
    WD_DISPATCH_FLAT(V.sp.flat, FL, WD_DISPATCH_PAIR(pw, pp, SW, SP, {
        launch_pdl(k_dot_part<SW, SP, true, FL>, grid, dim3(256), 0, c->st, (const void *)V.t, (const void *)V.s,
                   V.part, Vh, nrhs, V.bpr, (const BiState *)V.st);
        launch_pdl(k_scal_omega, dim3((nrhs + 127) / 128), dim3(128), 0, c->st, V.st, (const double *)V.part, nrhs,
                   V.bpr);
        XrUpdate<SW, SP, FL>::run(c, V, nrhs);
        launch_pdl(k_scal_beta, dim3(1), dim3(256), 0, c->st, V.st, (const double *)V.part, nrhs, V.bpr, V.count,
                   V.alist);
        launch_pdl(k_bicg_p<SW, SP, FL>, dim3(eb), dim3(256), 0, c->st, (const void *)V.r, V.p, (const void *)V.v,
                   (const BiState *)V.st, Vh, n);
    }));
    c->launches += 5;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int bicg_iter(wd_ctx *c, int pw, int pp, BiVecs &V, int nrhs) {
    WD_TRY(V.op(c, V.p, V.v, nrhs, V.op_user));       // v = A p
    WD_TRY(bicg_after_v(c, pw, pp, V, nrhs));
    WD_TRY(V.op(c, V.s, V.t, nrhs, V.op_user));       // t = A s
    return bicg_after_t(c, pw, pp, V, nrhs);
}

}  // namespace wd
