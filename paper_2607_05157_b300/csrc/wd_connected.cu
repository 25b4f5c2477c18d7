// Connected pseudoscalar two-point function with the two-level multigrid
// decomposition (Sec. 4, Eqs. 16-20 with L = 2):
//
//   G(t) = (1/T) sum_t' tr[D^{-1}(t+t', t') g5 D^{-1}(t', t+t') g5] = sum_ij G_ij(t),
//   B_1 = D^{-1} - P D_c^{-1} P^dag,   B_2 = P D_c^{-1} P^dag,
//   G_ij(t) = (1/T) sum_t' tr[B_i(t+t', t') g5 B_j(t', t+t') g5].
//
// Both level operators are gamma5-hermitian (P keeps the chirality halves
// apart), so G_ij(t) = (1/T) sum_t' tr[B_i(t+t', t') B_j(t+t', t')^dag], and
// with Rademacher noise eta on source timeslice t' and y_k = B_k eta
//   sample_ij(t) = (1/T) sum_t' sum_{x in t+t'} y_j(x)^dag y_i(x)
// is unbiased.  Level 1 (N1 samples, noise samples 0..N1-1): one fine solve
// and one coarse-corrected solve per (sample, t') give y_1 = D^{-1} eta - y_2,
// y_2 = P D_c^{-1} P^dag eta and the (1,1), (1,2), (2,1) samples.  The (2,2)
// term needs only coarse solves and is sampled on its own (N2 samples of the
// independent noise samples i | 2^21), so the variance of the total is
// var(S11 + S12 + S21)/N1 + var(S22)/N2.  The (2,2) term on the level-1
// noise comes for free and gives the plain (undecomposed) estimator
// |y_1 + y_2|^2 on the same samples, for comparison.
#include <math.h>
#include <string.h>

#include "wd_internal.h"

namespace wd {

int gen_time_diluted_eo(wd_ctx *c, uint64_t seed, int stream, int g0, int nb, double *be, double *bo, int *tsup);
int coarse_solve(wd_ctx *c, const double *b, double *x, int nrhs, double tol, int prec, int max_iter,
                 double *resid_out);
int auto_batch(wd_ctx *c, int total);

static constexpr int LEVEL2_STREAM = 1 << 21;

__global__ void k_sub_conn(double *z, const double *w, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) z[i] -= w[i];
}

// Partials over a chunk of timeslice tt (both parities) of one RHS:
// [0] |y1|^2, [1..2] y2^dag y1, [3] |y2|^2 (y1 nullable: level 2 only).
// grid (bps, nrhs, T); part[((r*T + tt)*bps + bx)*4 + q]
__global__ void k_contract_pairs(Geom g, const double *y1e, const double *y1o, const double *y2e, const double *y2o,
                                 double *part, int bps) {
    const int r = blockIdx.y, tt = blockIdx.z;
    const int slice = g.Vh / g.T;
    const int chunk = (2 * slice + bps - 1) / bps;
    const int u0 = blockIdx.x * chunk, u1 = min(u0 + chunk, 2 * slice);
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
        const int p = u >= slice, s = tt * slice + (u - p * slice);
        cx<double> v2[12];
        SIO<double>::load((const uint4 *)(p ? y2o : y2e) + (size_t)r * 12 * g.Vh, g.Vh, s, v2);
#pragma unroll
        for (int k = 0; k < 12; ++k) a[3] += v2[k].re * v2[k].re + v2[k].im * v2[k].im;
        if (y1e) {
            cx<double> v1[12];
            SIO<double>::load((const uint4 *)(p ? y1o : y1e) + (size_t)r * 12 * g.Vh, g.Vh, s, v1);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                a[0] += v1[k].re * v1[k].re + v1[k].im * v1[k].im;
                a[1] += v2[k].re * v1[k].re + v2[k].im * v1[k].im;     // conj(y2) y1
                a[2] += v2[k].re * v1[k].im - v2[k].im * v1[k].re;
            }
        }
    }
    __shared__ double sh[4][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        for (int o = 16; o > 0; o >>= 1) a[q] += __shfl_xor_sync(0xffffffffu, a[q], o);
        if (lane == 0) sh[q][wid] = a[q];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            double v = lane < nw ? sh[q][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) part[(((size_t)r * g.T + tt) * bps + blockIdx.x) * 4 + q] = v;
        }
    }
}

// S[sample][t] += (1/T) sum over the batch's RHS g = T*sample + t' of the
// partials at timeslice (t + t') mod T (fixed order).  S1: [N1][4][T][2]
// (pairs (1,1), (1,2), (2,1), (2,2)); S2: [N2][T][2].  level 1: S1, else S2.
__global__ void k_accumulate_pairs(const double *part, int bps, int T, int g0, int nb, int level, double *S1,
                                   double *S2, int s_first, int nsamp) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nsamp * T) return;
    const int si = s_first + idx / T, t = idx % T;
    const int a = max(g0, si * T), b = min(g0 + nb, (si + 1) * T);
    double q[4] = {0.0, 0.0, 0.0, 0.0};
    for (int gi = a; gi < b; ++gi) {
        const int tp = gi - si * T, tt = (t + tp) % T;
        const double *p = part + ((size_t)(gi - g0) * T + tt) * bps * 4;
        for (int k = 0; k < bps; ++k)
            for (int j = 0; j < 4; ++j) q[j] += p[4 * k + j];
    }
    const double w = 1.0 / T;
    if (level == 1) {
        double *o = S1 + (size_t)si * 4 * T * 2;
        o[(0 * T + t) * 2] += w * q[0];                      // (1,1): real
        o[(1 * T + t) * 2] += w * q[1];                      // (1,2) = y2^dag y1
        o[(1 * T + t) * 2 + 1] += w * q[2];
        o[(2 * T + t) * 2] += w * q[1];                      // (2,1) = conj(1,2)
        o[(2 * T + t) * 2 + 1] -= w * q[2];
        o[(3 * T + t) * 2] += w * q[3];                      // (2,2) on the level-1 noise
    } else {
        S2[((size_t)si * T + t) * 2] += w * q[3];
    }
}

// mean (mr, mi) and variance of the mean of N complex samples x_i = base[i * stride .. + 1]
__device__ void mean_var_of(const double *base, size_t stride, int N, double &mr, double &mi, double &v) {
    mr = 0.0; mi = 0.0; v = 0.0;
    for (int i = 0; i < N; ++i) { mr += base[i * stride]; mi += base[i * stride + 1]; }
    mr /= N; mi /= N;
    for (int i = 0; i < N; ++i) {
        const double dr = base[i * stride] - mr, di = base[i * stride + 1] - mi;
        v += dr * dr + di * di;
    }
    v = v / (N - 1) / N;
}

// G[6][T][2] and var[6][T]: pairs (1,1), (1,2), (2,1), (2,2) [from S2], the
// total (the level-1 per-sample sum of its three pairs plus the independent
// (2,2)) and the plain estimator (all four pairs on the level-1 noise)
__global__ void k_connected_stats(const double *S1, const double *S2, int N1, int N2, int T, double *G,
                                  double *var) {
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        for (int k = 0; k < 4; ++k) {
            double mr, mi, v;
            if (k < 3) mean_var_of(S1 + ((size_t)k * T + t) * 2, (size_t)4 * T * 2, N1, mr, mi, v);
            else mean_var_of(S2 + (size_t)t * 2, (size_t)T * 2, N2, mr, mi, v);
            G[(k * T + t) * 2] = mr;
            G[(k * T + t) * 2 + 1] = mi;
            var[k * T + t] = v;
        }
        for (int kind = 0; kind < 2; ++kind) {       // 0: level-1 sum of 3 pairs, 1: plain (4 pairs)
            const int np = kind == 0 ? 3 : 4;
            double sr = 0.0, si = 0.0, v1 = 0.0;
            for (int pass = 0; pass < 2; ++pass)
                for (int i = 0; i < N1; ++i) {
                    double xr = 0.0, xi = 0.0;
                    for (int q = 0; q < np; ++q) {
                        xr += S1[(((size_t)i * 4 + q) * T + t) * 2];
                        xi += S1[(((size_t)i * 4 + q) * T + t) * 2 + 1];
                    }
                    if (pass == 0) { sr += xr / N1; si += xi / N1; }
                    else v1 += (xr - sr) * (xr - sr) + (xi - si) * (xi - si);
                }
            if (kind == 0) {
                G[(4 * T + t) * 2] = sr + G[(3 * T + t) * 2];
                G[(4 * T + t) * 2 + 1] = si + G[(3 * T + t) * 2 + 1];
                var[4 * T + t] = v1 / (N1 - 1) / N1 + var[3 * T + t];
            } else {
                G[(5 * T + t) * 2] = sr;
                G[(5 * T + t) * 2 + 1] = si;
                var[5 * T + t] = v1 / (N1 - 1) / N1;
            }
        }
    }
}

}  // namespace wd

using namespace wd;

extern "C" int wd_connected_mlmc(wd_ctx *c, int N1, int N2, uint64_t seed, int prec, double tol, int batch,
                                 double *G, double *var, double *samples1, double *samples2, int64_t *n_solves_out) {
    if (!c || !G || !var || N1 < 2 || N2 < 2 || prec < 0 || prec > 2 || !(tol > 0)) {
        set_error("wd_connected_mlmc: bad argument (N1, N2 >= 2)");
        return WD_EINVAL;
    }
    if (!c->mg) { set_error("wd_connected_mlmc: needs wd_mg_setup"); return WD_EINVAL; }
    const Geom &g = c->g;
    const int T = g.T;
    if ((long)N1 * T > (1L << 30) || (long)N2 * T > (1L << 30)) { set_error("wd_connected_mlmc: too many samples"); return WD_EINVAL; }
    const long ncoarse = (long)c->mg->Vc * c->mg->ncd;
    double *S1, *S2, *Gd, *vd;
    WD_TRY(ws_get(c, "con.S1", sizeof(double) * 2 * 4 * (size_t)N1 * T, (void **)&S1));
    WD_TRY(ws_get(c, "con.S2", sizeof(double) * 2 * (size_t)N2 * T, (void **)&S2));
    WD_TRY(ws_get(c, "con.G", sizeof(double) * 2 * 6 * T, (void **)&Gd));
    WD_TRY(ws_get(c, "con.var", sizeof(double) * 6 * T, (void **)&vd));
    WD_CUDA(cudaMemsetAsync(S1, 0, sizeof(double) * 2 * 4 * (size_t)N1 * T, c->st));
    WD_CUDA(cudaMemsetAsync(S2, 0, sizeof(double) * 2 * (size_t)N2 * T, c->st));
    int64_t ns = 0;
    for (int level = 1; level <= 2; ++level) {
        const long total = (long)(level == 1 ? N1 : N2) * T;
        const int B = batch > 0 ? (int)(batch < total ? batch : total) : auto_batch(c, (int)total);
        for (long g0 = 0; g0 < total; g0 += B) {
            const int nb = (int)(total - g0 < B ? total - g0 : B);
            const size_t f = field_bytes(g, P64, nb);
            double *be, *bo, *ye, *yo, *we, *wo, *bc, *yc, *part;
            int *tsup;
            WD_TRY(ws_get(c, "con.be", f, (void **)&be));
            WD_TRY(ws_get(c, "con.bo", f, (void **)&bo));
            WD_TRY(ws_get(c, "con.we", f, (void **)&we));
            WD_TRY(ws_get(c, "con.wo", f, (void **)&wo));
            if (level == 1) {
                WD_TRY(ws_get(c, "con.ye", f, (void **)&ye));
                WD_TRY(ws_get(c, "con.yo", f, (void **)&yo));
            }
            WD_TRY(ws_get(c, "con.bc", sizeof(double2) * ncoarse * nb, (void **)&bc));
            WD_TRY(ws_get(c, "con.yc", sizeof(double2) * ncoarse * nb, (void **)&yc));
            WD_TRY(ws_get(c, "con.tsup", sizeof(int) * (size_t)nb, (void **)&tsup));
            int bps = (2 * (g.Vh / T) + 1023) / 1024;
            if (bps < 1) bps = 1;
            WD_TRY(ws_get(c, "con.part", sizeof(double) * 4 * (size_t)nb * T * bps, (void **)&part));
            WD_TRY(gen_time_diluted_eo(c, seed, level == 1 ? 0 : LEVEL2_STREAM, (int)g0, nb, be, bo, tsup));
            // y_2 = P D_c^{-1} P^dag eta
            WD_TRY(mg_restrict_eo(c, be, bo, bc, nb, true));
            int s = coarse_solve(c, bc, yc, nb, tol, prec, 100000, nullptr);
            if (s != WD_OK) return s;
            WD_TRY(mg_prolong_eo(c, yc, we, wo, nb, true));
            ns += nb;
            if (level == 1) {
                // y_1 = D^{-1} eta - y_2
                s = solve_eo(c, be, bo, ye, yo, nb, tol, prec, 100000, nullptr, nullptr, tsup);
                if (s != WD_OK) return s;
                const long nf = (long)nb * 24 * g.Vh;
                k_sub_conn<<<1184, 256, 0, c->st>>>(ye, we, nf);
                k_sub_conn<<<1184, 256, 0, c->st>>>(yo, wo, nf);
                c->launches += 2;
                ns += nb;
            }
            k_contract_pairs<<<dim3(bps, nb, T), 256, 0, c->st>>>(g, level == 1 ? ye : nullptr,
                                                                  level == 1 ? yo : nullptr, we, wo, part, bps);
            const int s_first = (int)(g0 / T), s_last = (int)((g0 + nb - 1) / T), nsamp = s_last - s_first + 1;
            k_accumulate_pairs<<<(nsamp * T + 127) / 128, 128, 0, c->st>>>(part, bps, T, (int)g0, nb, level, S1, S2,
                                                                           s_first, nsamp);
            c->launches += 2;
            WD_CUDA(cudaGetLastError());
        }
    }
    k_connected_stats<<<1, 128, 0, c->st>>>(S1, S2, N1, N2, T, Gd, vd);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    WD_CUDA(cudaMemcpyAsync(G, Gd, sizeof(double) * 2 * 6 * T, cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaMemcpyAsync(var, vd, sizeof(double) * 6 * T, cudaMemcpyDeviceToHost, c->st));
    if (samples1)
        WD_CUDA(cudaMemcpyAsync(samples1, S1, sizeof(double) * 2 * 4 * (size_t)N1 * T, cudaMemcpyDeviceToHost, c->st));
    if (samples2)
        WD_CUDA(cudaMemcpyAsync(samples2, S2, sizeof(double) * 2 * (size_t)N2 * T, cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaStreamSynchronize(c->st));
    WD_TRY(hop_err_check(c));
    if (n_solves_out) *n_solves_out = ns;
    return WD_OK;
}
