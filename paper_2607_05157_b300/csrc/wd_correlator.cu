// Pseudoscalar (pion) two-point correlator from point sources:
//   C(t) = sum_{x in t} sum_{s,a; s',a'} |D^{-1}(x, s, a; x0, s', a')|^2,
// the 12 columns of D^{-1} with a source at site x0 (one per spin-colour
// component), solved together as 12 right-hand sides.  With gamma5-hermiticity
// this is the connected pseudoscalar correlator sum_x tr[g5 S(x,x0) g5 S^dag]
// (the connected observable of Sec. 4 at a single source, without the
// multilevel splitting of Eqs. 16-20).
#include <vector>

#include "wd_internal.h"

namespace wd {

// b_k = unit vector on dof (x0, k), k = 0..11, as FP64 eo fields (zeroed by the
// caller); tsup[k] = the source timeslice (the Schur-source stencil skips the
// timeslices the source cannot reach)
__global__ void k_point_sources(double *be, double *bo, Geom g, int site0, int *tsup) {
    const int k = threadIdx.x;
    if (k >= 12) return;
    int x = site0 % g.X, r = site0 / g.X;
    int y = r % g.Y; r /= g.Y;
    int z = r % g.Z, t = r / g.Z;
    tsup[k] = t;
    const int p = (x + y + z + t) & 1, s = site0 >> 1;
    double2 *f = (double2 *)(p ? bo : be) + (size_t)k * 12 * g.Vh;
    f[(size_t)k * g.Vh + s] = make_double2(1.0, 0.0);
}

// part[(r*T + t)*bps + bx] = sum over a chunk of timeslice t of |x_r|^2 (both parities)
__global__ void k_norm_timeslice(Geom g, const double *xe, const double *xo, double *part, int bps) {
    const int r = blockIdx.y, t = blockIdx.z;
    const int slice = g.Vh / g.T;
    const int chunk = (2 * slice + bps - 1) / bps;
    const int u0 = blockIdx.x * chunk, u1 = min(u0 + chunk, 2 * slice);
    double acc = 0.0;
    for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
        const int p = u >= slice, s = t * slice + (u - p * slice);
        cx<double> v[12];
        SIO<double>::load((const uint4 *)(p ? xo : xe) + (size_t)r * 12 * g.Vh, g.Vh, s, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc += v[k].re * v[k].re + v[k].im * v[k].im;
    }
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sh[w];
        part[((size_t)r * g.T + t) * bps + blockIdx.x] = a;
    }
}

// C[t] = sum_r sum_b part[r][t][b], fixed order
__global__ void k_sum_correlator(const double *part, int nr, int T, int bps, double *C) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    double a = 0.0;
    for (int r = 0; r < nr; ++r)
        for (int b = 0; b < bps; ++b) a += part[((size_t)r * T + t) * bps + b];
    C[t] = a;
}

}  // namespace wd

using namespace wd;

extern "C" int wd_point_correlator(wd_ctx *c, const int src[4], int prec, double tol, double *C) {
    if (!c || !src || !C || prec < 0 || prec > 2 || !(tol > 0)) { set_error("wd_point_correlator: bad argument"); return WD_EINVAL; }
    const Geom &g = c->g;
    const int L[4] = {g.X, g.Y, g.Z, g.T};
    for (int m = 0; m < 4; ++m)
        if (src[m] < 0 || src[m] >= L[m]) { set_error("wd_point_correlator: source outside the lattice"); return WD_EINVAL; }
    const int site0 = src[0] + g.X * (src[1] + g.Y * (src[2] + g.Z * src[3]));
    const int nr = 12;
    const size_t f = field_bytes(g, P64, nr);
    double *be, *bo, *xe, *xo, *part, *Cd;
    int *tsup;
    WD_TRY(ws_get(c, "pc.tsup", sizeof(int) * nr, (void **)&tsup));
    WD_TRY(ws_get(c, "pc.be", f, (void **)&be));
    WD_TRY(ws_get(c, "pc.bo", f, (void **)&bo));
    WD_TRY(ws_get(c, "pc.xe", f, (void **)&xe));
    WD_TRY(ws_get(c, "pc.xo", f, (void **)&xo));
    int bps = (2 * (g.Vh / g.T) + 1023) / 1024;
    if (bps < 1) bps = 1;
    WD_TRY(ws_get(c, "pc.part", sizeof(double) * (size_t)nr * g.T * bps, (void **)&part));
    WD_TRY(ws_get(c, "pc.C", sizeof(double) * g.T, (void **)&Cd));
    WD_TRY(blas_zero(c, be, f));
    WD_TRY(blas_zero(c, bo, f));
    k_point_sources<<<1, 32, 0, c->st>>>(be, bo, g, site0, tsup);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    int s = solve_eo(c, be, bo, xe, xo, nr, tol, prec, 100000, nullptr, nullptr, tsup);
    if (s != WD_OK) return s;
    k_norm_timeslice<<<dim3(bps, nr, g.T), 256, 0, c->st>>>(g, xe, xo, part, bps);
    k_sum_correlator<<<(g.T + 127) / 128, 128, 0, c->st>>>(part, nr, g.T, bps, Cd);
    c->launches += 2;
    WD_CUDA(cudaGetLastError());
    WD_CUDA(cudaMemcpyAsync(C, Cd, sizeof(double) * g.T, cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaStreamSynchronize(c->st));
    return WD_OK;
}
