// Trace estimators: Hutchinson (Eq. 3) and stochastic probing
// with spin-colour / time dilution (Eqs. 13-14), estimating
// tr[B D^{-1}(t, t)] per timeslice with B = 1 or gamma5 (Eq. 21).
//
// The right-hand sides are never stored on the host and never read back:
//  * k_gen_rhs writes them straight into the FP64 eo fields from a counter
//    hash -- entry j = 12*site + 3*spin + colour of noise sample i is
//    1 - 2*topbit(splitmix64(seed ^ (i << 40) ^ j)) (Rademacher, Sec. 1),
//    masked to one colour c(x) = sum_j sigma_j x_j mod n_c of the torus
//    colouring (Eq. 15), one spin-colour component and/or one timeslice;
//  * k_contract regenerates the same entries while it forms
//    X(t) = sum_{x in t} conj(v(x)) (B D^{-1} v)(x) in FP64.
// Right-hand sides are enumerated sample-major, (sample, colour, component,
// timeslice), and solved in batches; per-sample values are accumulated in
// that fixed order, so results are deterministic.
#include <math.h>
#include <string.h>

#include <vector>

#include "wd_internal.h"

namespace wd {

struct EstParams {
    unsigned long long seed;
    int m;          // right-hand sides per sample
    int nc;         // colours (1 = no colour mask)
    int sigma[4];
    int dil;        // spin-colour dilution 1 or 12
    int TT;         // timeslices per sample (1 = no time dilution)
    int g0;         // global index of the first RHS of the batch
    int nrhs;       // RHS in this batch
    int gamma5;     // B = gamma5 (1) or 1 (0)
    int stream_hi;  // OR-ed into the noise sample index (separate noise streams; 0: the main one)
};

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Rademacher entry of dof j for noise sample `sample`
__device__ __forceinline__ double rademacher(unsigned long long seed, unsigned long long sample, unsigned long long j) {
    const unsigned long long h = splitmix64(seed ^ (sample << 40) ^ j);
    return (h >> 63) ? -1.0 : 1.0;
}

struct RhsDesc { int sample, colour, comp, tslice; };

__device__ __forceinline__ RhsDesc describe(const EstParams &P, int g) {
    RhsDesc d;
    d.sample = g / P.m;
    int j = g - d.sample * P.m;
    d.tslice = P.TT > 1 ? j % P.TT : -1;
    j /= P.TT;
    d.comp = P.dil > 1 ? j % P.dil : -1;
    j /= P.dil;
    d.colour = P.nc > 1 ? j : -1;
    return d;
}

// fills v[12] with the masked noise of site (x,y,z,t); returns false if the whole site is masked
__device__ __forceinline__ bool site_noise(const EstParams &P, const Geom &g, const RhsDesc &d, int x, int y, int z,
                                           int t, cx<double> v[12]) {
    bool on = true;
    if (d.tslice >= 0 && t != d.tslice) on = false;
    if (d.colour >= 0) {
        const long c = (long)P.sigma[0] * x + (long)P.sigma[1] * y + (long)P.sigma[2] * z + (long)P.sigma[3] * t;
        if ((int)(c % P.nc) != d.colour) on = false;
    }
    const unsigned long long site = (unsigned long long)(x + g.X * (y + g.Y * (z + (long)g.Z * t)));
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double e = 0.0;
        if (on && (d.comp < 0 || d.comp == k))
            e = rademacher(P.seed, (unsigned long long)(d.sample | P.stream_hi), 12ULL * site + k);
        v[k] = cmake(e, 0.0);
    }
    return on;
}

// b (FP64 eo, both parities) for the RHS of the batch
__global__ void k_gen_rhs(EstParams P, Geom g, double *be, double *bo) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)g.V * P.nrhs) return;
    const int r = (int)(i / g.V), site = (int)(i % g.V);
    int x = site % g.X, rr = site / g.X;
    int y = rr % g.Y; rr /= g.Y;
    int z = rr % g.Z, t = rr / g.Z;
    const RhsDesc d = describe(P, P.g0 + r);
    cx<double> v[12];
    site_noise(P, g, d, x, y, z, t, v);
    const int p = (x + y + z + t) & 1;
    SIO<double>::store((uint4 *)(p ? bo : be) + (size_t)r * 12 * g.Vh, g.Vh, site >> 1, v);
}

// partial X(rhs, t) over a chunk of timeslice t, both parities.
// grid (bps, nrhs, T); part[((rhs*T + t)*bps + bx)*2 + {re,im}]
__global__ void k_contract(EstParams P, Geom g, const double *xe, const double *xo, double *part, int bps) {
    const int r = blockIdx.y, t = blockIdx.z;
    const RhsDesc d = describe(P, P.g0 + r);
    const int slice = g.Vh / g.T;          // half-sites per timeslice and parity
    double are = 0.0, aim = 0.0;
    if (d.tslice < 0 || d.tslice == t) {
        const int chunk = (2 * slice + bps - 1) / bps;
        const int u0 = blockIdx.x * chunk, u1 = min(u0 + chunk, 2 * slice);
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
            const int p = u >= slice, s = t * slice + (u - p * slice);
            int x, y, z, tt;
            eo_coords(g, p, s, x, y, z, tt);
            cx<double> v[12];
            if (!site_noise(P, g, d, x, y, z, tt, v)) continue;
            cx<double> sol[12];
            SIO<double>::load((const uint4 *)(p ? xo : xe) + (size_t)r * 12 * g.Vh, g.Vh, s, sol);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const double sg = (P.gamma5 && k >= 6) ? -1.0 : 1.0;   // gamma5 = diag(1,1,-1,-1)
                // conj(v) * B sol with v real
                are += sg * v[k].re * sol[k].re;
                aim += sg * v[k].re * sol[k].im;
            }
        }
    }
    // block reduce
    __shared__ double sh[2][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        are += __shfl_xor_sync(0xffffffffu, are, o);
        aim += __shfl_xor_sync(0xffffffffu, aim, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { sh[0][wid] = are; sh[1][wid] = aim; }
    __syncthreads();
    if (wid == 0) {
        are = lane < nw ? sh[0][lane] : 0.0;
        aim = lane < nw ? sh[1][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            are += __shfl_xor_sync(0xffffffffu, are, o);
            aim += __shfl_xor_sync(0xffffffffu, aim, o);
        }
        if (lane == 0) {
            double *q = part + (((size_t)r * g.T + t) * bps + blockIdx.x) * 2;
            q[0] = are;
            q[1] = aim;
        }
    }
}

// Support timeslice of each RHS of the batch (-1: all timeslices), for the
// stencil of the Schur source
__global__ void k_tsup(EstParams P, int *tsup) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < P.nrhs) tsup[r] = describe(P, P.g0 + r).tslice;
}

// B = gamma5 with time dilution: every RHS eta lives on one timeslice t0 and
// X(t0) = eta^dag g5 x over both parities.  With x_o = eta_o + k H_oe x_e and
// the gamma5-hermiticity H_oe^dag g5 = g5 H_eo of the hop,
//   eta_o^dag g5 x_o = eta_o^dag g5 eta_o + k (H_eo eta_o)^dag g5 x_e,
// and k H_eo eta_o = bhat_e - eta_e, so
//   X(t0) = bhat_e^dag g5 x_e + eta_o^dag g5 eta_o
// (exact algebra: the odd solution is never formed).  bhat_e lives on the
// timeslices t0 - 1, t0, t0 + 1.  grid (bps, nrhs, 3), z = t - t0 + 1;
// part[((rhs*3 + z)*bps + bx)*2 + {re,im}]
__global__ void k_contract_schur(EstParams P, Geom g, const double *bhat, const double *xe, double *part, int bps) {
    const int r = blockIdx.y, z3 = blockIdx.z;
    const RhsDesc d = describe(P, P.g0 + r);
    const int T = g.T;
    const int t = (d.tslice + z3 - 1 + T) % T;
    const int slice = g.Vh / T;            // half-sites per timeslice and parity
    double are = 0.0, aim = 0.0;
    if (!(T == 2 && z3 == 2)) {            // T = 2: t0 - 1 and t0 + 1 coincide
        const int chunk = (slice + bps - 1) / bps;
        const int u0 = blockIdx.x * chunk, u1 = min(u0 + chunk, slice);
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
            const int s = t * slice + u;
            cx<double> bv[12], xv[12];
            SIO<double>::load((const uint4 *)bhat + (size_t)r * 12 * g.Vh, g.Vh, s, bv);
            SIO<double>::load((const uint4 *)xe + (size_t)r * 12 * g.Vh, g.Vh, s, xv);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const double sg = k >= 6 ? -1.0 : 1.0;
                are += sg * (bv[k].re * xv[k].re + bv[k].im * xv[k].im);
                aim += sg * (bv[k].re * xv[k].im - bv[k].im * xv[k].re);
            }
            if (z3 == 1) {                 // eta_o^dag g5 eta_o on the odd sites of t0
                int x, y, zz, tt;
                eo_coords(g, 1, s, x, y, zz, tt);
                cx<double> v[12];
                if (site_noise(P, g, d, x, y, zz, tt, v)) {
#pragma unroll
                    for (int k = 0; k < 12; ++k) are += (k >= 6 ? -1.0 : 1.0) * v[k].re * v[k].re;
                }
            }
        }
    }
    __shared__ double sh[2][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        are += __shfl_xor_sync(0xffffffffu, are, o);
        aim += __shfl_xor_sync(0xffffffffu, aim, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { sh[0][wid] = are; sh[1][wid] = aim; }
    __syncthreads();
    if (wid == 0) {
        are = lane < nw ? sh[0][lane] : 0.0;
        aim = lane < nw ? sh[1][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            are += __shfl_xor_sync(0xffffffffu, are, o);
            aim += __shfl_xor_sync(0xffffffffu, aim, o);
        }
        if (lane == 0) {
            double *q = part + (((size_t)r * 3 + z3) * bps + blockIdx.x) * 2;
            q[0] = are;
            q[1] = aim;
        }
    }
}

// X[sample][t] += sum over this batch's RHS of that sample on timeslice t of
// their k_contract_schur partials (fixed order)
__global__ void k_accumulate_schur(EstParams P, int T, const double *part, int bps, double *X, int first_sample,
                                   int nsamples) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nsamples * T) return;
    const int si = first_sample + idx / T, t = idx % T;
    const int a = max(P.g0, si * P.m), b = min(P.g0 + P.nrhs, (si + 1) * P.m);
    double re = 0.0, im = 0.0;
    for (int gidx = a; gidx < b; ++gidx) {
        if (describe(P, gidx).tslice != t) continue;
        const double *q = part + (size_t)(gidx - P.g0) * 3 * bps * 2;
        for (int k = 0; k < 3 * bps; ++k) { re += q[2 * k]; im += q[2 * k + 1]; }
    }
    X[((size_t)si * T + t) * 2] += re;
    X[((size_t)si * T + t) * 2 + 1] += im;
}

// X[sample][t] += sum over this batch's RHS of that sample (fixed order)
__global__ void k_accumulate(EstParams P, int T, const double *part, int bps, double *X, int first_sample,
                             int nsamples) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nsamples * T) return;
    const int si = first_sample + idx / T, t = idx % T;
    const int a = max(P.g0, si * P.m), b = min(P.g0 + P.nrhs, (si + 1) * P.m);
    double re = 0.0, im = 0.0;
    for (int gidx = a; gidx < b; ++gidx) {
        const double *q = part + ((size_t)(gidx - P.g0) * T + t) * bps * 2;
        for (int k = 0; k < bps; ++k) { re += q[2 * k]; im += q[2 * k + 1]; }
    }
    X[((size_t)si * T + t) * 2] += re;
    X[((size_t)si * T + t) * 2 + 1] += im;
}

// mean and sample variance per timeslice and of the total over timeslices.
// out_mean[2*(T+1)], out_var[T+1]
// sum of v over the block (blockDim.x a power of two <= 256), fixed tree order;
// every thread gets the result
__device__ double block_sum_fixed(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// per-timeslice and total means and sample variances of X [N][T][2]: one
// thread per timeslice column; the total (sum over t of each sample) with the
// samples spread over the block and block sums in a fixed order
__global__ void k_mean_var(const double *X, int N, int T, double *out_mean, double *out_var) {
    __shared__ double sh[256];
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        double mr = 0, mi = 0;
        for (int i = 0; i < N; ++i) { mr += X[((size_t)i * T + t) * 2]; mi += X[((size_t)i * T + t) * 2 + 1]; }
        mr /= N; mi /= N;
        double v = 0;
        for (int i = 0; i < N; ++i) {
            const double xr = X[((size_t)i * T + t) * 2] - mr, xi = X[((size_t)i * T + t) * 2 + 1] - mi;
            v += xr * xr + xi * xi;
        }
        out_mean[2 * t] = mr;
        out_mean[2 * t + 1] = mi;
        out_var[t] = N > 1 ? v / (N - 1) : NAN;
    }
    double sr = 0, si = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        for (int u = 0; u < T; ++u) { sr += X[((size_t)i * T + u) * 2]; si += X[((size_t)i * T + u) * 2 + 1]; }
    const double mr = block_sum_fixed(sr, sh) / N, mi = block_sum_fixed(si, sh) / N;
    double v = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double xr = 0, xi = 0;
        for (int u = 0; u < T; ++u) { xr += X[((size_t)i * T + u) * 2]; xi += X[((size_t)i * T + u) * 2 + 1]; }
        v += (xr - mr) * (xr - mr) + (xi - mi) * (xi - mi);
    }
    v = block_sum_fixed(v, sh);
    if (threadIdx.x == 0) {
        out_mean[2 * T] = mr;
        out_mean[2 * T + 1] = mi;
        out_var[T] = N > 1 ? v / (N - 1) : NAN;
    }
}

// Solve + contract a sample-major range of right-hand sides, accumulating into
// X (device, [N][T][2]).  Used by every estimator.
int estimate_rhs_range(wd_ctx *c, EstParams P, int total, int batch, double tol, int prec, double *X, int64_t *nsolves) {
    const Geom &g = c->g;
    const int T = g.T;
    for (int g0 = 0; g0 < total; g0 += batch) {
        const int nb = min(batch, total - g0);
        P.g0 = g0;
        P.nrhs = nb;
        const size_t f = field_bytes(g, P64, nb);
        double *be, *bo, *xe, *xo, *part;
        WD_TRY(ws_get(c, "est.be", f, (void **)&be));
        WD_TRY(ws_get(c, "est.bo", f, (void **)&bo));
        WD_TRY(ws_get(c, "est.xe", f, (void **)&xe));
        WD_TRY(ws_get(c, "est.xo", f, (void **)&xo));
        const int slice2 = 2 * (g.Vh / T);
        int bps = (slice2 + 1023) / 1024;
        if (bps < 1) bps = 1;
        WD_TRY(ws_get(c, "est.part", sizeof(double) * 2 * (size_t)nb * (T > 3 ? T : 3) * bps, (void **)&part));
        const long n = (long)g.V * nb;
        k_gen_rhs<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>(P, g, be, bo);
        c->launches++;
        WD_CUDA(cudaGetLastError());
        // time dilution: each source lives on one timeslice (the Schur-source
        // stencil skips the sites it cannot reach); with B = gamma5 the
        // contraction uses bhat and the even solution only (k_contract_schur)
        int *tsup = nullptr;
        if (P.TT > 1) {
            WD_TRY(ws_get(c, "est.tsup", sizeof(int) * (size_t)nb, (void **)&tsup));
            k_tsup<<<(nb + 127) / 128, 128, 0, c->st>>>(P, tsup);
            c->launches++;
            WD_CUDA(cudaGetLastError());
        }
        const bool schur = P.TT > 1 && P.gamma5;
        const double *bhat = nullptr;
        int s = solve_eo(c, be, bo, xe, schur ? nullptr : xo, nb, tol, prec, 100000, nullptr, nullptr, tsup, &bhat);
        if (s != WD_OK) return s;
        const int s_first = g0 / P.m, s_last = (g0 + nb - 1) / P.m;
        const int ns = s_last - s_first + 1;
        if (schur) {
            const int bps1 = ((g.Vh / T) + 1023) / 1024;
            k_contract_schur<<<dim3(bps1, nb, 3), 256, 0, c->st>>>(P, g, bhat, xe, part, bps1);
            k_accumulate_schur<<<(ns * T + 127) / 128, 128, 0, c->st>>>(P, T, part, bps1, X, s_first, ns);
        } else {
            k_contract<<<dim3(bps, nb, T), 256, 0, c->st>>>(P, g, xe, xo, part, bps);
            k_accumulate<<<(ns * T + 127) / 128, 128, 0, c->st>>>(P, T, part, bps, X, s_first, ns);
        }
        c->launches += 2;
        WD_CUDA(cudaGetLastError());
        *nsolves += nb;
    }
    return WD_OK;
}

int auto_batch(wd_ctx *c, int total) {
    // FP64 eo fields of the estimator and the solver (~14 half-fields) plus the
    // FP32 Krylov vectors (8 half-fields) per RHS; keep the batch under ~96 GB
    // (a third of the GPU's memory)
    const double per = (double)c->g.Vh * (14 * 192.0 + 8 * 96.0);
    int b = (int)(96e9 / per);
    if (b > 384) b = 384;
    if (b < 1) b = 1;
    return b < total ? b : total;
}

int finish_estimate(wd_ctx *c, const double *X, int N, double *estimate, double *sample_var, double *samples_out) {
    const int T = c->g.T;
    double *mean, *var;
    WD_TRY(ws_get(c, "est.mean", sizeof(double) * 2 * (T + 1), (void **)&mean));
    WD_TRY(ws_get(c, "est.var", sizeof(double) * (T + 1), (void **)&var));
    k_mean_var<<<1, 256, 0, c->st>>>(X, N, T, mean, var);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    WD_CUDA(cudaMemcpyAsync(estimate, mean, sizeof(double) * 2 * (T + 1), cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaMemcpyAsync(sample_var, var, sizeof(double) * (T + 1), cudaMemcpyDeviceToHost, c->st));
    if (samples_out)
        WD_CUDA(cudaMemcpyAsync(samples_out, X, sizeof(double) * 2 * (size_t)N * T, cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaStreamSynchronize(c->st));
    return WD_OK;
}

int mlmc2_estimate(wd_ctx *c, int N1, int N2, uint64_t seed, int gamma5, int prec, int batch, double tol,
                   double *estimate, double *sample_var, int64_t *nsolves, double *samples_out,
                   int (*level1)(wd_ctx *, void *, int, int, double, int, double *, int64_t *) = nullptr,
                   void *level1_user = nullptr, const CoarseProbe *cp = nullptr);
int coarse_solve(wd_ctx *c, const double *b, double *x, int nrhs, double tol, int prec, int max_iter,
                 double *resid_out);

__global__ void k_sub_fields(double *z, const double *w, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) z[i] -= w[i];
}

// Level 1 of the two-level estimator with probing (WD_MLMC2_PROBE, Sec. 6
// outlook): for the probing x dilution (x timeslice) vectors v of N1 noise
// samples, X1(t) += sum_{x in t} conj(v) B (D^{-1} v - P D_c^{-1} P^dag v),
// v regenerated by the contraction from the counter hash.  u: EstParams.
static int level1_probe(wd_ctx *c, void *u, int N1, int batch, double tol, int prec, double *X1, int64_t *ns) {
    EstParams P = *(const EstParams *)u;
    const Geom &g = c->g;
    const int T = g.T;
    const long total = (long)N1 * P.m;
    const long ncoarse = (long)c->mg->Vc * c->mg->ncd;
    const int B = batch > 0 ? (int)(batch < total ? batch : total) : auto_batch(c, (int)total);
    for (long g0 = 0; g0 < total; g0 += B) {
        const int nb = (int)(total - g0 < B ? total - g0 : B);
        P.g0 = (int)g0;
        P.nrhs = nb;
        const size_t f = field_bytes(g, P64, nb);
        double *be, *bo, *ze, *zo, *we, *wo, *bc, *yc, *part;
        WD_TRY(ws_get(c, "mlp.be", f, (void **)&be));
        WD_TRY(ws_get(c, "mlp.bo", f, (void **)&bo));
        WD_TRY(ws_get(c, "mlp.ze", f, (void **)&ze));
        WD_TRY(ws_get(c, "mlp.zo", f, (void **)&zo));
        WD_TRY(ws_get(c, "mlp.we", f, (void **)&we));
        WD_TRY(ws_get(c, "mlp.wo", f, (void **)&wo));
        WD_TRY(ws_get(c, "mlp.bc", sizeof(double2) * ncoarse * nb, (void **)&bc));
        WD_TRY(ws_get(c, "mlp.yc", sizeof(double2) * ncoarse * nb, (void **)&yc));
        int bps = (2 * (g.Vh / T) + 1023) / 1024;
        if (bps < 1) bps = 1;
        WD_TRY(ws_get(c, "mlp.part", sizeof(double) * 2 * (size_t)nb * T * bps, (void **)&part));
        const long n = (long)g.V * nb;
        k_gen_rhs<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>(P, g, be, bo);
        c->launches++;
        WD_CUDA(cudaGetLastError());
        int *tsup = nullptr;
        if (P.TT > 1) {
            WD_TRY(ws_get(c, "mlp.tsup", sizeof(int) * (size_t)nb, (void **)&tsup));
            k_tsup<<<(nb + 127) / 128, 128, 0, c->st>>>(P, tsup);
            c->launches++;
        }
        int s = solve_eo(c, be, bo, ze, zo, nb, tol, prec, 100000, nullptr, nullptr, tsup);
        if (s != WD_OK) return s;
        WD_TRY(mg_restrict_eo(c, be, bo, bc, nb, true));
        s = coarse_solve(c, bc, yc, nb, tol, prec, 100000, nullptr);
        if (s != WD_OK) return s;
        WD_TRY(mg_prolong_eo(c, yc, we, wo, nb, true));
        const long nf = (long)nb * 24 * g.Vh;
        k_sub_fields<<<1184, 256, 0, c->st>>>(ze, we, nf);
        k_sub_fields<<<1184, 256, 0, c->st>>>(zo, wo, nf);
        const int s_first = (int)(g0 / P.m), s_last = (int)((g0 + nb - 1) / P.m);
        const int nsamp = s_last - s_first + 1;
        k_contract<<<dim3(bps, nb, T), 256, 0, c->st>>>(P, g, ze, zo, part, bps);
        k_accumulate<<<(nsamp * T + 127) / 128, 128, 0, c->st>>>(P, T, part, bps, X1, s_first, nsamp);
        c->launches += 4;
        WD_CUDA(cudaGetLastError());
        *ns += 2 * (int64_t)nb;
    }
    return WD_OK;
}

// Rademacher noise of samples [sample0, sample0 + nrhs) (no masks) into FP64 eo fields
int gen_noise_eo(wd_ctx *c, uint64_t seed, int sample0, int nrhs, double *be, double *bo) {
    EstParams P;
    memset(&P, 0, sizeof(P));
    P.seed = seed; P.m = 1; P.nc = 1; P.dil = 1; P.TT = 1; P.g0 = sample0; P.nrhs = nrhs;
    const long n = (long)c->g.V * nrhs;
    k_gen_rhs<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>(P, c->g, be, bo);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// Sign words of the plain Rademacher noise gen_noise_eo writes:
// bits[(p Vh + s) 12 + k] has bit r set where entry k of half-site s of parity
// p is -1 in sample sample0 + r (r < nrhs <= 64).  The same hash as
// site_noise, so the words describe exactly the fields of gen_noise_eo.
__global__ void k_noise_signs(EstParams P, Geom g, unsigned long long *bits) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)g.V * 12) return;
    const int k = (int)(i % 12);
    const long eo = i / 12;
    const int p = (int)(eo / g.Vh), s = (int)(eo - (long)p * g.Vh);
    int x, y, z, t;
    eo_coords(g, p, s, x, y, z, t);
    const unsigned long long site = (unsigned long long)(x + g.X * (y + g.Y * (z + (long)g.Z * t)));
    unsigned long long w = 0;
    for (int r = 0; r < P.nrhs; ++r) {
        const RhsDesc d = describe(P, P.g0 + r);
        if (rademacher(P.seed, (unsigned long long)(d.sample | P.stream_hi), 12ULL * site + k) < 0.0) w |= 1ULL << r;
    }
    bits[i] = w;
}

int gen_noise_signs(wd_ctx *c, uint64_t seed, int sample0, int nrhs, unsigned long long *bits) {
    if (nrhs < 1 || nrhs > 64) { set_error("noise signs: 1..64 samples per word"); return WD_EINVAL; }
    EstParams P;
    memset(&P, 0, sizeof(P));
    P.seed = seed; P.m = 1; P.nc = 1; P.dil = 1; P.TT = 1; P.g0 = sample0; P.nrhs = nrhs;
    const long n = (long)c->g.V * 12;
    k_noise_signs<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>(P, c->g, bits);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// X[sample0 + r][t] += sum_{x in t} conj(eta_r(x)) (B y_r)(x) for unmasked
// Rademacher noise of samples sample0 + r (r < nrhs); X is [N][T][2]
int contract_noise_eo(wd_ctx *c, uint64_t seed, int sample0, int nrhs, int gamma5, const double *ye,
                      const double *yo, double *X) {
    EstParams P;
    memset(&P, 0, sizeof(P));
    P.seed = seed; P.m = 1; P.nc = 1; P.dil = 1; P.TT = 1; P.g0 = sample0; P.nrhs = nrhs; P.gamma5 = gamma5;
    const Geom &g = c->g;
    int bps = (2 * (g.Vh / g.T) + 1023) / 1024;
    if (bps < 1) bps = 1;
    double *part;
    WD_TRY(ws_get(c, "est.part", sizeof(double) * 2 * (size_t)nrhs * g.T * bps, (void **)&part));
    k_contract<<<dim3(bps, nrhs, g.T), 256, 0, c->st>>>(P, g, ye, yo, part, bps);
    k_accumulate<<<(nrhs * g.T + 127) / 128, 128, 0, c->st>>>(P, g.T, part, bps, X, sample0, nrhs);
    c->launches += 2;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// Time-diluted Rademacher sources: RHS g = T * i + t' (g0 <= g < g0 + nb) is
// noise sample i | stream on timeslice t' only, into FP64 eo fields; tsup[r]
// = t' (device, nb entries) for the Schur-source stencil
int gen_time_diluted_eo(wd_ctx *c, uint64_t seed, int stream, int g0, int nb, double *be, double *bo, int *tsup) {
    EstParams P;
    memset(&P, 0, sizeof(P));
    P.seed = seed; P.nc = 1; P.dil = 1; P.TT = c->g.T; P.m = c->g.T; P.g0 = g0; P.nrhs = nb; P.stream_hi = stream;
    const long n = (long)c->g.V * nb;
    k_gen_rhs<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>(P, c->g, be, bo);
    k_tsup<<<(nb + 127) / 128, 128, 0, c->st>>>(P, tsup);
    c->launches += 2;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// Estimator parameters for Hutchinson / probing with the given dilution
int est_params(wd_ctx *c, int method, int dilution, int d, uint64_t seed, int gamma5, EstParams &P) {
    memset(&P, 0, sizeof(P));
    const int dil = dilution & 0xff;
    if (dil != 1 && dil != 12) { set_error("dilution must be 1 or 12 (optionally | WD_DIL_TIME)"); return WD_EINVAL; }
    P.seed = seed;
    P.dil = dil;
    P.TT = (dilution & WD_DIL_TIME) ? c->g.T : 1;
    P.gamma5 = gamma5;
    P.nc = 1;
    if (method == WD_PROBE) {
        // 4D colouring, or (WD_COLOR_3D, time-diluted only) the colouring of
        // one timeslice: sigma_t = 0, every timeslice coloured alike
        const bool c3 = (dilution & WD_COLOR_3D) != 0;
        if (c3 && !(dilution & WD_DIL_TIME)) {
            set_error("WD_COLOR_3D needs time dilution (WD_DIL_TIME)");
            return WD_EINVAL;
        }
        int nc = 0, sig[4] = {0, 0, 0, 0};
        const int s = probe_color(c->dims, c3 ? 3 : 4, d, &nc, sig, nullptr);
        if (s != WD_OK) { set_error("no torus colouring for distance %d", d); return s; }
        P.nc = nc;
        for (int j = 0; j < 4; ++j) P.sigma[j] = j < (c3 ? 3 : 4) ? sig[j] : 0;
    }
    P.m = P.nc * P.dil * P.TT;
    return WD_OK;
}

// RHS [g0, g0 + nrhs) of the sample-major enumeration into FP64 eo fields
// (nrhs = 0: only report the RHS count per sample)
int gen_masked_eo(wd_ctx *c, int method, int dilution, int d, uint64_t seed, int g0, int nrhs, double *be,
                  double *bo, int *per_sample) {
    EstParams P;
    WD_TRY(est_params(c, method, dilution, d, seed, 0, P));
    *per_sample = P.m;
    if (nrhs <= 0) return WD_OK;
    P.g0 = g0;
    P.nrhs = nrhs;
    const long n = (long)c->g.V * nrhs;
    k_gen_rhs<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>(P, c->g, be, bo);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

}  // namespace wd

using namespace wd;

extern "C" int trace_estimate(wd_ctx *c, int method, int dilution, int N, int n2, int d, uint64_t seed, int op,
                              int prec, int batch, double tol, double *estimate, double *sample_var,
                              int64_t *n_solves_out, double *samples_out) {
    if (!c || !estimate || !sample_var || N < 1 || prec < 0 || prec > 2 || !(tol > 0) || (op != 0 && op != 1)) {
        set_error("trace_estimate: bad argument");
        return WD_EINVAL;
    }
    if ((dilution & 0xff) != 1 && (dilution & 0xff) != 12) {
        set_error("trace_estimate: dilution must be 1 or 12 (optionally | WD_DIL_TIME)");
        return WD_EINVAL;
    }
    int64_t ns = 0;
    if (method == WD_MLMC2 || method == WD_MLMC2_PROBE) {
        if (n2 < 1) { set_error("trace_estimate: MLMC2 needs n2 >= 1"); return WD_EINVAL; }
        if (!c->mg) { set_error("trace_estimate: MLMC2 needs wd_mg_setup"); return WD_EINVAL; }
        int s;
        if (method == WD_MLMC2_PROBE) {
            EstParams P;
            WD_TRY(est_params(c, WD_PROBE, dilution, d, seed, op == WD_TR_G5_DINV, P));
            if ((long)N * P.m > (1L << 30)) { set_error("trace_estimate: too many right-hand sides"); return WD_EINVAL; }
            s = mlmc2_estimate(c, N, n2, seed, op, prec, batch, tol, estimate, sample_var, &ns, samples_out,
                               level1_probe, &P);
        } else {
            s = mlmc2_estimate(c, N, n2, seed, op, prec, batch, tol, estimate, sample_var, &ns, samples_out);
        }
        if (n_solves_out) *n_solves_out = ns;
        return s;
    }
    if (method != WD_HUTCH && method != WD_PROBE) { set_error("trace_estimate: unknown method %d", method); return WD_EINVAL; }
    EstParams P;
    WD_TRY(est_params(c, method, dilution, d, seed, op == WD_TR_G5_DINV, P));
    const long total = (long)N * P.m;
    if (total > (1L << 30)) { set_error("trace_estimate: too many right-hand sides"); return WD_EINVAL; }
    const int T = c->g.T;
    double *X;
    WD_TRY(ws_get(c, "est.X", sizeof(double) * 2 * (size_t)N * T, (void **)&X));
    WD_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * 2 * (size_t)N * T, c->st));
    const int b = batch > 0 ? (int)(batch < total ? batch : total) : auto_batch(c, (int)total);
    int s = estimate_rhs_range(c, P, (int)total, b, tol, prec, X, &ns);
    if (n_solves_out) *n_solves_out = ns;
    if (s != WD_OK) return s;
    return finish_estimate(c, X, N, estimate, sample_var, samples_out);
}

extern "C" int trace_estimate_mlmc_probe(wd_ctx *c, int dilution, int d, int N1, int coarse_dil, int d2, int N2,
                                         uint64_t seed, int op, int prec, int batch, double tol, double *estimate,
                                         double *sample_var, int64_t *n_solves_out, double *samples1,
                                         double *samples2) {
    if (!c || !estimate || !sample_var || N1 < 1 || N2 < 1 || prec < 0 || prec > 2 || !(tol > 0) ||
        (op != 0 && op != 1) || d2 < 0) {
        set_error("trace_estimate_mlmc_probe: bad argument");
        return WD_EINVAL;
    }
    if (!c->mg) { set_error("trace_estimate_mlmc_probe: needs wd_mg_setup"); return WD_EINVAL; }
    const int ncd = c->mg->ncd;
    if (coarse_dil != 1 && coarse_dil != ncd) {
        set_error("trace_estimate_mlmc_probe: coarse dilution must be 1 or the %d coarse dofs of a site", ncd);
        return WD_EINVAL;
    }
    EstParams P;
    WD_TRY(est_params(c, WD_PROBE, dilution, d, seed, op == WD_TR_G5_DINV, P));
    if ((long)N1 * P.m > (1L << 30)) { set_error("trace_estimate_mlmc_probe: too many right-hand sides"); return WD_EINVAL; }
    CoarseProbe cp;
    memset(&cp, 0, sizeof(cp));
    for (int j = 0; j < 4; ++j) cp.cd[j] = c->mg->cd[j];
    cp.nc = 1;
    if (d2 > 0) {
        int sig[4];
        WD_TRY(probe_color(c->mg->cd, 4, d2, &cp.nc, sig, nullptr));
        for (int j = 0; j < 4; ++j) cp.sigma[j] = sig[j];
    }
    cp.dil = coarse_dil;
    cp.m = cp.nc * cp.dil;
    if ((long)N2 * cp.m > (1L << 30)) { set_error("trace_estimate_mlmc_probe: too many coarse vectors"); return WD_EINVAL; }
    int64_t ns = 0;
    const int s = mlmc2_estimate(c, N1, N2, seed, op, prec, batch, tol, estimate, sample_var, &ns, samples1,
                                 level1_probe, &P, &cp);
    if (n_solves_out) *n_solves_out = ns;
    if (s != WD_OK) return s;
    if (samples2) memcpy(samples2, c->last_level2.data(), sizeof(double) * 2 * (size_t)N2 * c->g.T);
    return WD_OK;
}
