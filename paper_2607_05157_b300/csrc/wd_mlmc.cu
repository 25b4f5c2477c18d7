// Two-level multigrid multilevel Monte Carlo (Sec. 2, Eqs. 9-12 with L = 2)
// and the GPU test-vector setup.
//
// tr(B D^{-1}) = tr(B M_1) + tr(B P D_c^{-1} P^dag), M_1 = D^{-1} - P D_c^{-1} P^dag.
// Level 1, N_1 fine Rademacher samples eta:
//   X_1(t) = sum_{x in t} eta^dag B (D^{-1} eta - P D_c^{-1} P^dag eta)
// Level 2, N_2 coarse Rademacher samples xi (coarse dof j = ncd*X + i, noise
// sample | 2^23):   X_2(t) = sum_{x in t} (P xi)^dag B (P D_c^{-1} xi),
// an unbiased estimate of tr(P^dag B(t) P D_c^{-1}) = tr(B(t) P D_c^{-1} P^dag)
// (for B = 1 it is xi^dag D_c^{-1} xi since P^dag P = I).
// The estimate is mean(X_1) + mean(X_2), its variance s_1^2/N_1 + s_2^2/N_2.
#include <math.h>
#include <string.h>

#include <vector>

#include "wd_internal.h"

namespace wd {

int gen_noise_eo(wd_ctx *c, uint64_t seed, int sample0, int nrhs, double *be, double *bo);
int contract_noise_eo(wd_ctx *c, uint64_t seed, int sample0, int nrhs, int gamma5, const double *ye,
                      const double *yo, double *X);
int coarse_solve(wd_ctx *c, const double *b, double *x, int nrhs, double tol, int prec, int max_iter,
                 double *resid_out);
Space coarse_space(wd_ctx *c);
int auto_batch(wd_ctx *c, int total);
int finish_estimate(wd_ctx *c, const double *X, int N, double *estimate, double *sample_var, double *samples_out);

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// coarse Rademacher noise: xi[r][j] for samples (sample0 + r) | 2^23
__global__ void k_coarse_noise(double2 *xi, unsigned long long seed, int sample0, long ncoarse, int nrhs) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= ncoarse * nrhs) return;
    const unsigned long long r = (unsigned long long)(i / ncoarse), j = (unsigned long long)(i % ncoarse);
    const unsigned long long sample = ((unsigned long long)sample0 + r) | (1ULL << 23);
    const unsigned long long h = mix64(seed ^ (sample << 40) ^ j);
    xi[i] = make_double2((h >> 63) ? -1.0 : 1.0, 0.0);
}

// coarse probing noise: RHS g = g0 + r of the sample-major enumeration (m
// vectors per sample: colour j / dil, coarse dof j % dil) is the coarse
// Rademacher noise of sample (g / m) | 2^23 masked to the sites of that
// colour and (dil > 1) that dof of the site
__global__ void k_coarse_noise_probe(double2 *xi, unsigned long long seed, int g0, long ncoarse, int nrhs, int ncd,
                                     CoarseProbe cp) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= ncoarse * nrhs) return;
    const int r = (int)(i / ncoarse);
    const long idx = i % ncoarse;
    const int g = g0 + r, sample = g / cp.m, j = g % cp.m;
    const int comp = cp.dil > 1 ? j % cp.dil : -1, colour = j / cp.dil;
    const int X = (int)(idx / ncd), k = (int)(idx % ncd);
    int x = X % cp.cd[0], q = X / cp.cd[0];
    const int y = q % cp.cd[1];
    q /= cp.cd[1];
    const int z = q % cp.cd[2], t = q / cp.cd[2];
    const long cval = (long)cp.sigma[0] * x + (long)cp.sigma[1] * y + (long)cp.sigma[2] * z + (long)cp.sigma[3] * t;
    double v = 0.0;
    if ((int)(cval % cp.nc) == colour && (comp < 0 || comp == k)) {
        const unsigned long long h = mix64(seed ^ ((((unsigned long long)sample) | (1ULL << 23)) << 40) ^
                                           (unsigned long long)idx);
        v = (h >> 63) ? -1.0 : 1.0;
    }
    xi[i] = make_double2(v, 0.0);
}

// X[(g0 + r) T + t] -= part[r][t] (complex), one RHS per sample
__global__ void k_sub_part(double *X, const double *part, int g0, int nrhs, int T) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrhs * T) return;
    X[((size_t)g0 * T + i) * 2] -= part[(size_t)i * 2];
    X[((size_t)g0 * T + i) * 2 + 1] -= part[(size_t)i * 2 + 1];
}

// partial X(rhs, t) = sum_{x in t} conj(a(x)) (B b)(x) for explicit eo fields a, b
__global__ void k_contract_fields(Geom g, const double *ae, const double *ao, const double *be, const double *bo,
                                  int gamma5, double *part, int bps) {
    const int r = blockIdx.y, t = blockIdx.z;
    const int slice = g.Vh / g.T;
    const int chunk = (2 * slice + bps - 1) / bps;
    const int u0 = blockIdx.x * chunk, u1 = min(u0 + chunk, 2 * slice);
    double are = 0.0, aim = 0.0;
    for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
        const int p = u >= slice, s = t * slice + (u - p * slice);
        cx<double> va[12], vb[12];
        SIO<double>::load((const uint4 *)(p ? ao : ae) + (size_t)r * 12 * g.Vh, g.Vh, s, va);
        SIO<double>::load((const uint4 *)(p ? bo : be) + (size_t)r * 12 * g.Vh, g.Vh, s, vb);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double sg = (gamma5 && k >= 6) ? -1.0 : 1.0;
            are += sg * (va[k].re * vb[k].re + va[k].im * vb[k].im);
            aim += sg * (va[k].re * vb[k].im - va[k].im * vb[k].re);
        }
    }
    __shared__ double sh[2][32];
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

// X[sample][t] += sum over the batch's RHS g = g0 + r of that sample (g / m
// == sample, m vectors per sample) of sum_k part[r][t][k]; fixed order
__global__ void k_accumulate_fields(int T, const double *part, int bps, double *X, int g0, int nrhs, int m) {
    const int s_first = g0 / m, nsamp = (g0 + nrhs - 1) / m - s_first + 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nsamp * T) return;
    const int si = s_first + idx / T, t = idx % T;
    const int a = max(g0, si * m), b = min(g0 + nrhs, (si + 1) * m);
    double re = 0, im = 0;
    for (int gi = a; gi < b; ++gi) {
        const double *q = part + ((size_t)(gi - g0) * T + t) * bps * 2;
        for (int k = 0; k < bps; ++k) { re += q[2 * k]; im += q[2 * k + 1]; }
    }
    X[((size_t)si * T + t) * 2] += re;
    X[((size_t)si * T + t) * 2 + 1] += im;
}

// three levels: estimate = sum of the means, variance = sum var_l / N_l
__global__ void k_mlmc_combine3(const double *m1, const double *v1, const double *m2, const double *v2,
                                const double *m3, const double *v3, int N1, int N2, int N3, int n, double *mean,
                                double *var) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        mean[2 * t] = m1[2 * t] + m2[2 * t] + m3[2 * t];
        mean[2 * t + 1] = m1[2 * t + 1] + m2[2 * t + 1] + m3[2 * t + 1];
        var[t] = v1[t] / N1 + v2[t] / N2 + v3[t] / N3;
    }
}

// estimate = mean_1 + mean_2, variance = var_1 / N1 + var_2 / N2
__global__ void k_mlmc_combine(const double *m1, const double *v1, const double *m2, const double *v2, int N1, int N2,
                               int n, double *mean, double *var) {
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        mean[2 * t] = m1[2 * t] + m2[2 * t];
        mean[2 * t + 1] = m1[2 * t + 1] + m2[2 * t + 1];
        var[t] = v1[t] / N1 + v2[t] / N2;
    }
}

static int contract_fields(wd_ctx *c, const double *ae, const double *ao, const double *be, const double *bo,
                           int gamma5, int nrhs, double *X, int g0, int m = 1) {
    const Geom &g = c->g;
    int bps = (2 * (g.Vh / g.T) + 1023) / 1024;
    if (bps < 1) bps = 1;
    double *part;
    WD_TRY(ws_get(c, "mlmc.part", sizeof(double) * 2 * (size_t)nrhs * g.T * bps, (void **)&part));
    k_contract_fields<<<dim3(bps, nrhs, g.T), 256, 0, c->st>>>(g, ae, ao, be, bo, gamma5, part, bps);
    k_accumulate_fields<<<(nrhs * g.T + 127) / 128, 128, 0, c->st>>>(g.T, part, bps, X, g0, nrhs, m);
    c->launches += 2;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

static int mean_var_dev(wd_ctx *c, const double *X, int N, double *mean, double *var);

// entry points of this file's kernels for the three-level estimator (wd_mg3.cu)
int mlmc_contract_fields(wd_ctx *c, const double *ae, const double *ao, const double *be, const double *bo,
                         int gamma5, int nrhs, double *X, int sample0) {
    return contract_fields(c, ae, ao, be, bo, gamma5, nrhs, X, sample0, 1);
}
int mlmc_mean_var(wd_ctx *c, const double *X, int N, double *mean, double *var) {
    return mean_var_dev(c, X, N, mean, var);
}
int coarse_noise_dev(wd_ctx *c, double *xi, uint64_t seed, int sample0, long ncoarse, int nrhs) {
    const long n = ncoarse * nrhs;
    k_coarse_noise<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>((double2 *)xi, seed, sample0, ncoarse, nrhs);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}
int mlmc_combine3(wd_ctx *c, const double *m1, const double *v1, const double *m2, const double *v2,
                  const double *m3, const double *v3, int N1, int N2, int N3, double *mean, double *var);

// level1 (nullable): fills X1 [N1][T][2] and adds its solves to *ns in place
// of the plain Rademacher level 1 (WD_MLMC2_PROBE passes the probing one)
int mlmc2_estimate(wd_ctx *c, int N1, int N2, uint64_t seed, int gamma5, int prec, int batch, double tol,
                   double *estimate, double *sample_var, int64_t *nsolves, double *samples_out,
                   int (*level1)(wd_ctx *, void *, int, int, double, int, double *, int64_t *), void *level1_user,
                   const CoarseProbe *cp) {
    if (!c->mg) { set_error("trace_estimate: MLMC2 needs wd_mg_setup"); return WD_EINVAL; }
    const Geom &g = c->g;
    const int T = g.T;
    const long ncoarse = (long)c->mg->Vc * c->mg->ncd;
    const int B = batch > 0 ? batch : auto_batch(c, N1 > N2 ? N1 : N2);
    double *X1, *X2;
    WD_TRY(ws_get(c, "mlmc.X1", sizeof(double) * 2 * (size_t)N1 * T, (void **)&X1));
    WD_TRY(ws_get(c, "mlmc.X2", sizeof(double) * 2 * (size_t)N2 * T, (void **)&X2));
    WD_CUDA(cudaMemsetAsync(X1, 0, sizeof(double) * 2 * (size_t)N1 * T, c->st));
    WD_CUDA(cudaMemsetAsync(X2, 0, sizeof(double) * 2 * (size_t)N2 * T, c->st));
    int64_t ns = 0;
    // ---- level 1: eta^dag B (D^{-1} - P D_c^{-1} P^dag) eta
    if (level1) WD_TRY(level1(c, level1_user, N1, batch, tol, prec, X1, &ns));
    for (int s0 = 0; s0 < (level1 ? 0 : N1); s0 += B) {
        const int nb = N1 - s0 < B ? N1 - s0 : B;
        const size_t f = field_bytes(g, P64, nb);
        double *be, *bo, *ze, *zo, *bc, *yc;
        WD_TRY(ws_get(c, "mlmc.be", f, (void **)&be));
        WD_TRY(ws_get(c, "mlmc.bo", f, (void **)&bo));
        WD_TRY(ws_get(c, "mlmc.ze", f, (void **)&ze));
        WD_TRY(ws_get(c, "mlmc.zo", f, (void **)&zo));
        WD_TRY(ws_get(c, "mlmc.bc", sizeof(double2) * ncoarse * nb, (void **)&bc));
        WD_TRY(ws_get(c, "mlmc.yc", sizeof(double2) * ncoarse * nb, (void **)&yc));
        WD_TRY(gen_noise_eo(c, seed, s0, nb, be, bo));
        int s = solve_eo(c, be, bo, ze, zo, nb, tol, prec, 100000, nullptr, nullptr);
        if (s != WD_OK) return s;
        // P^dag eta, kept per timeslice of each aggregate (Rt) for the coarse contraction
        double *Rt, *part;
        WD_TRY(ws_get(c, "mlmc.rt", sizeof(double2) * ncoarse * c->mg->agg[3] * nb, (void **)&Rt));
        WD_TRY(ws_get(c, "mlmc.part", sizeof(double) * 2 * (size_t)nb * T, (void **)&part));
        WD_TRY(mg_restrict_t_noise(c, seed, s0, be, bo, Rt, bc, nb));
        s = coarse_solve(c, bc, yc, nb, tol, prec, 100000, nullptr);
        if (s != WD_OK) return s;
        // X_1(t) = eta^dag B z - sum_{x in t} eta^dag B (P y): the first on the
        // fine lattice, the second on the coarse one from Rt (no prolongation)
        WD_TRY(contract_noise_eo(c, seed, s0, nb, gamma5, ze, zo, X1));
        WD_TRY(mg_contract_rt(c, Rt, yc, gamma5, nb, part));
        k_sub_part<<<(nb * T + 127) / 128, 128, 0, c->st>>>(X1, part, s0, nb, T);
        c->launches++;
        WD_CUDA(cudaGetLastError());
        ns += 2 * nb;
    }
    // ---- level 2: (P xi)^dag B (P D_c^{-1} xi), xi plain coarse noise or
    // (cp) the coarse probing vectors of each sample
    const int mc = cp ? cp->m : 1;          // coarse vectors per level-2 sample
    const long total2 = (long)N2 * mc;
    // level 2 holds coarse fields only (~24 per RHS in the coarse solve): up to ~32 GB of them per batch
    long cb = (long)(32e9 / ((double)ncoarse * 16.0 * 24.0));
    if (cb < 1) cb = 1;
    const int B2 = batch > 0 ? (int)(batch < total2 ? batch : total2)
                             : (int)(total2 < cb ? total2 : (cb < (1L << 30) ? cb : (1L << 30)));
    for (long s0l = 0; s0l < total2; s0l += B2) {
        const int s0 = (int)s0l;
        const int nb = (int)(total2 - s0l < B2 ? total2 - s0l : B2);
        double *xi, *yc;
        WD_TRY(ws_get(c, "mlmc.bc", sizeof(double2) * ncoarse * nb, (void **)&xi));
        WD_TRY(ws_get(c, "mlmc.yc", sizeof(double2) * ncoarse * nb, (void **)&yc));
        const long n = ncoarse * nb;
        if (cp)
            k_coarse_noise_probe<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>((double2 *)xi, seed, s0, ncoarse,
                                                                                 nb, c->mg->ncd, *cp);
        else
            k_coarse_noise<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>((double2 *)xi, seed, s0, ncoarse, nb);
        c->launches++;
        WD_CUDA(cudaGetLastError());
        int s = coarse_solve(c, xi, yc, nb, tol, prec, 100000, nullptr);
        if (s != WD_OK) return s;
        // X_2(t) = sum_{x in t} (P xi)^dag B (P y)(x), contracted on the coarse
        // lattice with the per-timeslice Gram matrices of P (no fine fields)
        double *part;
        WD_TRY(ws_get(c, "mlmc.part", sizeof(double) * 2 * (size_t)nb * T, (void **)&part));
        WD_TRY(mg_contract_coarse_t(c, xi, yc, gamma5, nb, part));
        k_accumulate_fields<<<(nb * T + 127) / 128, 128, 0, c->st>>>(T, part, 1, X2, s0, nb, mc);
        c->launches++;
        WD_CUDA(cudaGetLastError());
        ns += nb;
    }
    double *m1, *v1, *m2, *v2, *mean, *var;
    WD_TRY(ws_get(c, "mlmc.m1", sizeof(double) * 2 * (T + 1), (void **)&m1));
    WD_TRY(ws_get(c, "mlmc.v1", sizeof(double) * (T + 1), (void **)&v1));
    WD_TRY(ws_get(c, "mlmc.m2", sizeof(double) * 2 * (T + 1), (void **)&m2));
    WD_TRY(ws_get(c, "mlmc.v2", sizeof(double) * (T + 1), (void **)&v2));
    WD_TRY(ws_get(c, "mlmc.mean", sizeof(double) * 2 * (T + 1), (void **)&mean));
    WD_TRY(ws_get(c, "mlmc.var", sizeof(double) * (T + 1), (void **)&var));
    WD_TRY(mean_var_dev(c, X1, N1, m1, v1));
    WD_TRY(mean_var_dev(c, X2, N2, m2, v2));
    k_mlmc_combine<<<1, 128, 0, c->st>>>(m1, v1, m2, v2, N1, N2, T + 1, mean, var);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    WD_CUDA(cudaMemcpyAsync(estimate, mean, sizeof(double) * 2 * (T + 1), cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaMemcpyAsync(sample_var, var, sizeof(double) * (T + 1), cudaMemcpyDeviceToHost, c->st));
    if (samples_out)
        WD_CUDA(cudaMemcpyAsync(samples_out, X1, sizeof(double) * 2 * (size_t)N1 * T, cudaMemcpyDeviceToHost, c->st));
    c->last_level2.resize((size_t)2 * N2 * T);
    WD_CUDA(cudaMemcpyAsync(c->last_level2.data(), X2, sizeof(double) * 2 * (size_t)N2 * T, cudaMemcpyDeviceToHost,
                            c->st));
    c->last_n2 = N2;
    WD_CUDA(cudaStreamSynchronize(c->st));
    *nsolves = ns;
    return WD_OK;
}

// Mean and unbiased variance over the N samples of each timeslice t < T and of
// their sum over t (t = T): one warp per t, lanes over the samples (lane l
// takes l, l + 32, ...), combined by a fixed butterfly.
__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__global__ void k_mean_var2(const double *X, int N, int T, double *out_mean, double *out_var) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int t = blockIdx.x * nw + (threadIdx.x >> 5);
    if (t > T) return;
    auto sample = [&](int i, double &xr, double &xi) {
        xr = 0; xi = 0;
        if (t < T) { xr = X[((size_t)i * T + t) * 2]; xi = X[((size_t)i * T + t) * 2 + 1]; }
        else for (int u = 0; u < T; ++u) { xr += X[((size_t)i * T + u) * 2]; xi += X[((size_t)i * T + u) * 2 + 1]; }
    };
    double mr = 0, mi = 0;
    for (int i = lane; i < N; i += 32) {
        double xr, xi;
        sample(i, xr, xi);
        mr += xr;
        mi += xi;
    }
    mr = warp_sum_d(mr) / N;
    mi = warp_sum_d(mi) / N;
    double v = 0;
    for (int i = lane; i < N; i += 32) {
        double xr, xi;
        sample(i, xr, xi);
        v += (xr - mr) * (xr - mr) + (xi - mi) * (xi - mi);
    }
    v = warp_sum_d(v);
    if (lane == 0) {
        out_mean[2 * t] = mr;
        out_mean[2 * t + 1] = mi;
        out_var[t] = N > 1 ? v / (N - 1) : 0.0;
    }
}

static int mean_var_dev(wd_ctx *c, const double *X, int N, double *mean, double *var) {
    const int T = c->g.T;
    k_mean_var2<<<(T + 1 + 7) / 8, 256, 0, c->st>>>(X, N, T, mean, var);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// ---- test vectors: tv_iters inverse iterations v <- D^{-1} v / |v| from Rademacher starts
__global__ void k_scale_by(double *f, const double *n2a, const double *n2b, long per_rhs, int nrhs) {
    const long n = per_rhs * nrhs;
    int rc = -1;
    double sc = 0.0;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int r = (int)(i / per_rhs);
        if (r != rc) { rc = r; sc = 1.0 / sqrt(n2a[r] + n2b[r]); }   // once per vector a thread enters
        f[i] *= sc;
    }
}

int mg_generate_tv(wd_ctx *c, int nv, int iters, uint64_t seed, double *tv_dev) {
    const Geom &g = c->g;
    const size_t f = field_bytes(g, P64, nv);
    double *ve, *vo, *xe, *xo, *n2;
    WD_TRY(ws_get(c, "tv.ve", f, (void **)&ve));
    WD_TRY(ws_get(c, "tv.vo", f, (void **)&vo));
    WD_TRY(ws_get(c, "tv.xe", f, (void **)&xe));
    WD_TRY(ws_get(c, "tv.xo", f, (void **)&xo));
    WD_TRY(ws_get(c, "tv.n2", sizeof(double) * 2 * nv, (void **)&n2));
    WD_TRY(gen_noise_eo(c, seed, 1 << 22, nv, ve, vo));
    const Space sp = fine_space(g);
    for (int it = 0; it < iters; ++it) {
        // an approximate inverse suffices here: the FP32 solve to 1e-6
        int s = solve_eo_fp32(c, ve, vo, xe, xo, nv, 1e-6);
        if (s != WD_OK) return s;
        WD_TRY(blas_norm2(c, sp, P64, xe, nv, n2));
        WD_TRY(blas_norm2(c, sp, P64, xo, nv, n2 + nv));
        const long per = 24L * g.Vh;
        k_scale_by<<<1184, 256, 0, c->st>>>(xe, n2, n2 + nv, per, nv);
        k_scale_by<<<1184, 256, 0, c->st>>>(xo, n2, n2 + nv, per, nv);
        c->launches += 2;
        std::swap(ve, xe);
        std::swap(vo, xo);
    }
    return eo_to_user(c, ve, vo, P64, tv_dev, true, nv);
}

}  // namespace wd

using namespace wd;

extern "C" int wd_mg_test_vectors(wd_ctx *c, int nv, int iters, uint64_t seed, double *tv_out) {
    if (!c || nv < 1 || iters < 0 || !tv_out) {
        set_error("wd_mg_test_vectors: bad argument");
        return WD_EINVAL;
    }
    WD_TRY(mg_generate_tv(c, nv, iters, seed, tv_out));
    WD_CUDA(cudaStreamSynchronize(c->st));
    return WD_OK;
}

extern "C" int wd_mlmc_level2_samples(wd_ctx *c, double *samples_out, int n2) {
    if (!c || !samples_out || n2 != c->last_n2) { set_error("wd_mlmc_level2_samples: no matching MLMC2 estimate"); return WD_EINVAL; }
    memcpy(samples_out, c->last_level2.data(), sizeof(double) * c->last_level2.size());
    return WD_OK;
}

namespace wd {
int mlmc_combine3(wd_ctx *c, const double *m1, const double *v1, const double *m2, const double *v2,
                  const double *m3, const double *v3, int N1, int N2, int N3, double *mean, double *var) {
    k_mlmc_combine3<<<1, 128, 0, c->st>>>(m1, v1, m2, v2, m3, v3, N1, N2, N3, c->g.T + 1, mean, var);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}
}  // namespace wd
