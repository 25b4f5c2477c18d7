// Derivatives of the trace estimates.  The paper has no gradients;
// they follow from differentiating its quadratic forms X = v^dag B D^{-1} v:
//   dX = - w^dag (dD) z,   z = D^{-1} v,   w = D^{-dag} B^dag v.
// gamma5-hermiticity, D^{-dag} = g5 D^{-1} g5, turns the adjoint solve into an
// ordinary one: w = g5 D^{-1} (g5 B v).  For B = g5 * diag(g(t)) with equal
// weights g this is w = g g5 z: no second solve at all.
// Link force: for U_mu(x) -> U_mu(x) + h Delta,
//   d/dh (-w^dag dD z) = tr(Delta G) + conj(tr(Delta H)),
//   G_mu(x) = kappa b sum_s z(x+mu)_s [(1-g_mu) w(x)]_s^dag,
//   H_mu(x) = kappa b sum_s [(1+g_mu) w(x+mu)]_s z(x)_s^dag,
// b = bc[mu] on links that wrap around the lattice.  kappa: since
// dD/dkappa = (D - 1)/kappa, dX/dkappa = (w^dag z - X) / kappa.
#include <math.h>
#include <string.h>

#include <vector>

#include "wd_internal.h"

namespace wd {

// out = (1 + sign*g_mu) w, chiral basis g_mu = [[0, A], [A^dag, 0]]
template <int MU>
__device__ __forceinline__ void one_pm_gamma(const cx<double> w[12], double sign, cx<double> o[12]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cx<double> w0 = w[c], w1 = w[3 + c], w2 = w[6 + c], w3 = w[9 + c];
        cx<double> a0, a1, b0, b1;   // A (w2, w3) and A^dag (w0, w1)
        if (MU == 0)      { a0 = times_mi(w3); a1 = times_mi(w2); b0 = times_i(w1); b1 = times_i(w0); }
        else if (MU == 1) { a0 = cmake(-w3.re, -w3.im); a1 = w2; b0 = w1; b1 = cmake(-w0.re, -w0.im); }
        else if (MU == 2) { a0 = times_mi(w2); a1 = times_i(w3); b0 = times_i(w0); b1 = times_mi(w1); }
        else              { a0 = w2; a1 = w3; b0 = w0; b1 = w1; }
        o[c] = w0 + sign * a0;
        o[3 + c] = w1 + sign * a1;
        o[6 + c] = w2 + sign * b0;
        o[9 + c] = w3 + sign * b1;
    }
}

template <int MU>
__device__ __forceinline__ void force_dir(const Geom &g, int x, int y, int z, int t, int p, int s, const double *we,
                                          const double *wo, const double *ze, const double *zo, int nrhs,
                                          cx<double> G[9], cx<double> H[9]) {
    int c[4] = {x, y, z, t};
    const int L[4] = {g.X, g.Y, g.Z, g.T};
    c[MU] = c[MU] + 1 == L[MU] ? 0 : c[MU] + 1;
    const int sp = (c[0] + g.X * (c[1] + g.Y * (c[2] + g.Z * c[3]))) >> 1;
    const double *wx = p ? wo : we, *zx = p ? zo : ze, *wn = p ? we : wo, *zn = p ? ze : zo;
    for (int r = 0; r < nrhs; ++r) {
        cx<double> a[12], b[12], q[12];
        const size_t off = (size_t)r * 12 * g.Vh;
        SIO<double>::load((const uint4 *)(wx + 2 * off), g.Vh, s, a);
        one_pm_gamma<MU>(a, -1.0, q);                      // (1 - g) w(x)
        SIO<double>::load((const uint4 *)(zn + 2 * off), g.Vh, sp, b);   // z(x+mu)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int sg = 0; sg < 4; ++sg) cfma_conj(G[3 * i + j], q[3 * sg + j], b[3 * sg + i]);
        SIO<double>::load((const uint4 *)(wn + 2 * off), g.Vh, sp, a);   // w(x+mu)
        one_pm_gamma<MU>(a, +1.0, q);                      // (1 + g) w(x+mu)
        SIO<double>::load((const uint4 *)(zx + 2 * off), g.Vh, s, b);    // z(x)
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int sg = 0; sg < 4; ++sg) cfma_conj(H[3 * i + j], b[3 * sg + j], q[3 * sg + i]);
    }
}

// G, H [4][V][9] complex (lexicographic) += scale * kappa * b * force of the nrhs eo field pairs
__global__ void k_force(Geom g, int4 bc, double kscale, const double *we, const double *wo, const double *ze,
                        const double *zo, int nrhs, double2 *G, double2 *H, int accumulate) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= 4L * g.V) return;
    const int mu = (int)(i / g.V), site = (int)(i % g.V);
    int x = site % g.X, r = site / g.X;
    int y = r % g.Y; r /= g.Y;
    int z = r % g.Z, t = r / g.Z;
    const int p = (x + y + z + t) & 1, s = site >> 1;
    cx<double> Gm[9], Hm[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) { Gm[k] = cmake(0.0, 0.0); Hm[k] = cmake(0.0, 0.0); }
    if (mu == 0) force_dir<0>(g, x, y, z, t, p, s, we, wo, ze, zo, nrhs, Gm, Hm);
    else if (mu == 1) force_dir<1>(g, x, y, z, t, p, s, we, wo, ze, zo, nrhs, Gm, Hm);
    else if (mu == 2) force_dir<2>(g, x, y, z, t, p, s, we, wo, ze, zo, nrhs, Gm, Hm);
    else force_dir<3>(g, x, y, z, t, p, s, we, wo, ze, zo, nrhs, Gm, Hm);
    const int cc[4] = {x, y, z, t}, L[4] = {g.X, g.Y, g.Z, g.T}, bv[4] = {bc.x, bc.y, bc.z, bc.w};
    const double f = kscale * (cc[mu] == L[mu] - 1 ? bv[mu] : 1);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double2 gv = make_double2(f * Gm[k].re, f * Gm[k].im), hv = make_double2(f * Hm[k].re, f * Hm[k].im);
        const size_t o = (size_t)i * 9 + k;
        if (accumulate) { gv.x += G[o].x; gv.y += G[o].y; hv.x += H[o].x; hv.y += H[o].y; }
        G[o] = gv;
        H[o] = hv;
    }
}

// out = (g5 if gamma5) * diag(wt[t(x)]) * in on FP64 eo fields (both parities)
__global__ void k_weight_g5(Geom g, const double *in_e, const double *in_o, double *out_e, double *out_o,
                            const double *wt, int gamma5, int nrhs) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= 2L * g.Vh * nrhs) return;
    const int r = (int)(i / (2L * g.Vh));
    const int rem = (int)(i % (2L * g.Vh));
    const int p = rem >= g.Vh, s = rem - p * g.Vh;
    int x, y, z, t;
    eo_coords(g, p, s, x, y, z, t);
    const size_t off = (size_t)r * 12 * g.Vh;
    cx<double> v[12];
    SIO<double>::load((const uint4 *)((p ? in_o : in_e) + 2 * off), g.Vh, s, v);
    const double wgt = wt[t];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double sg = (gamma5 && k >= 6) ? -wgt : wgt;
        v[k] = sg * v[k];
    }
    SIO<double>::store((uint4 *)((p ? out_o : out_e) + 2 * off), g.Vh, s, v);
}

// per-RHS partial sums of conj(a).b over both parities of FP64 eo fields
__global__ void k_dot_eo(const double *ae, const double *ao, const double *be, const double *bo, long per, int nrhs,
                         double *out) {
    // one block per RHS, deterministic order
    const int r = blockIdx.x;
    double re = 0, im = 0;
    for (long u = threadIdx.x; u < 2 * per; u += blockDim.x) {
        const int p = u >= per;
        const long k = u - p * per;
        const double2 a = ((const double2 *)(p ? ao : ae))[(size_t)r * per + k];
        const double2 b = ((const double2 *)(p ? bo : be))[(size_t)r * per + k];
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
    }
    __shared__ double sh[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = re; sh[1][threadIdx.x >> 5] = im; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sh[0][w]; b += sh[1][w]; }
        out[2 * r] = a;
        out[2 * r + 1] = b;
    }
}

int force_eo(wd_ctx *c, const double *we, const double *wo, const double *ze, const double *zo, int nrhs,
             double scale, double *G, double *H, int accumulate) {
    const int4 bc = make_int4(c->bc[0], c->bc[1], c->bc[2], c->bc[3]);
    const long n = 4L * c->g.V;
    int slot;
    // algorithmic bytes: w, z at x and x+mu per link and RHS, G and H written once
    prof_begin(c, WD_K_FORCE, (double)n * (nrhs * 4.0 * 192.0 + 2 * 144.0), &slot);
    k_force<<<(unsigned)((n + 127) / 128), 128, 0, c->st>>>(c->g, bc, scale * c->kappa, we, wo, ze, zo, nrhs,
                                                            (double2 *)G, (double2 *)H, accumulate);
    prof_end(c, slot);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// exposed by wd_estim.cu
int gen_masked_eo(wd_ctx *c, int method, int dilution, int d, uint64_t seed, int g0, int nrhs, double *be,
                  double *bo, int *per_sample);

}  // namespace wd

using namespace wd;

extern "C" int wd_link_force(wd_ctx *c, const double *w, const double *z, int nrhs, double *G, double *H,
                             int accumulate) {
    if (!c || nrhs < 0 || !G || !H || ((!w || !z) && nrhs > 0)) { set_error("wd_link_force: bad argument"); return WD_EINVAL; }
    const size_t f = field_bytes(c->g, P64, nrhs > 0 ? nrhs : 1);
    double *we, *wo, *ze, *zo;
    WD_TRY(ws_get(c, "force.we", f, (void **)&we));
    WD_TRY(ws_get(c, "force.wo", f, (void **)&wo));
    WD_TRY(ws_get(c, "force.ze", f, (void **)&ze));
    WD_TRY(ws_get(c, "force.zo", f, (void **)&zo));
    if (nrhs > 0) {
        WD_TRY(user_to_eo(c, w, true, P64, we, wo, nrhs));
        WD_TRY(user_to_eo(c, z, true, P64, ze, zo, nrhs));
    }
    WD_TRY(force_eo(c, we, wo, ze, zo, nrhs, 1.0, G, H, accumulate));
    WD_CUDA(cudaStreamSynchronize(c->st));
    return WD_OK;
}

extern "C" int trace_gradient(wd_ctx *c, int method, int dilution, int N, int d, uint64_t seed, int op, int prec,
                              int batch, double tol, const double *weights, double *dkappa, double *G, double *H) {
    if (!c || !G || !H || !dkappa || N < 1 || (op != 0 && op != 1) || prec < 0 || prec > 2 || !(tol > 0) ||
        (method != WD_HUTCH && method != WD_PROBE)) {
        set_error("trace_gradient: bad argument");
        return WD_EINVAL;
    }
    const Geom &g = c->g;
    const int T = g.T;
    std::vector<double> wt(T, 1.0);
    if (weights) for (int t = 0; t < T; ++t) wt[t] = weights[t];
    bool uniform = true;
    for (int t = 1; t < T; ++t) uniform = uniform && wt[t] == wt[0];
    double *wt_d;
    WD_TRY(ws_get(c, "grad.wt", sizeof(double) * T, (void **)&wt_d));
    WD_CUDA(cudaMemcpyAsync(wt_d, wt.data(), sizeof(double) * T, cudaMemcpyHostToDevice, c->st));
    int m = 0;
    WD_TRY(gen_masked_eo(c, method, dilution, d, seed, 0, 0, nullptr, nullptr, &m));   // RHS per sample
    const long total = (long)N * m;
    int B = batch > 0 ? batch : 64;
    if (B > total) B = (int)total;
    const double scale = 1.0 / N;
    double dk_re = 0.0;
    bool first = true;
    for (long g0 = 0; g0 < total; g0 += B) {
        const int nb = (int)(total - g0 < B ? total - g0 : B);
        const size_t f = field_bytes(g, P64, nb);
        double *ve, *vo, *ze, *zo, *se, *so, *we, *wo, *dots;
        WD_TRY(ws_get(c, "grad.ve", f, (void **)&ve));
        WD_TRY(ws_get(c, "grad.vo", f, (void **)&vo));
        WD_TRY(ws_get(c, "grad.ze", f, (void **)&ze));
        WD_TRY(ws_get(c, "grad.zo", f, (void **)&zo));
        WD_TRY(ws_get(c, "grad.se", f, (void **)&se));
        WD_TRY(ws_get(c, "grad.so", f, (void **)&so));
        WD_TRY(ws_get(c, "grad.we", f, (void **)&we));
        WD_TRY(ws_get(c, "grad.wo", f, (void **)&wo));
        WD_TRY(ws_get(c, "grad.dots", sizeof(double) * 4 * nb, (void **)&dots));
        WD_TRY(gen_masked_eo(c, method, dilution, d, seed, (int)g0, nb, ve, vo, &m));
        int s = solve_eo(c, ve, vo, ze, zo, nb, tol, prec, 100000, nullptr, nullptr);
        if (s != WD_OK) return s;
        const unsigned eb = (unsigned)((2L * g.Vh * nb + 255) / 256);
        // s = B v = g5^op diag(wt) v  (B is Hermitian and real here)
        k_weight_g5<<<eb, 256, 0, c->st>>>(g, ve, vo, se, so, wt_d, op, nb);
        c->launches++;
        if (op == 1 && uniform) {
            // w = D^{-dag} g5 wt v = wt g5 D^{-1} v = wt g5 z
            std::vector<double> one(T, wt[0]);
            WD_CUDA(cudaMemcpyAsync(wt_d, one.data(), sizeof(double) * T, cudaMemcpyHostToDevice, c->st));
            k_weight_g5<<<eb, 256, 0, c->st>>>(g, ze, zo, we, wo, wt_d, 1, nb);
            WD_CUDA(cudaMemcpyAsync(wt_d, wt.data(), sizeof(double) * T, cudaMemcpyHostToDevice, c->st));
            c->launches++;
        } else {
            // w = g5 D^{-1} (g5 B v): one ordinary solve per RHS
            double *ue, *uo;
            WD_TRY(ws_get(c, "grad.ue", f, (void **)&ue));
            WD_TRY(ws_get(c, "grad.uo", f, (void **)&uo));
            std::vector<double> one(T, 1.0);
            double *one_d;
            WD_TRY(ws_get(c, "grad.one", sizeof(double) * T, (void **)&one_d));
            WD_CUDA(cudaMemcpyAsync(one_d, one.data(), sizeof(double) * T, cudaMemcpyHostToDevice, c->st));
            k_weight_g5<<<eb, 256, 0, c->st>>>(g, se, so, ue, uo, one_d, 1, nb);       // g5 B v
            s = solve_eo(c, ue, uo, we, wo, nb, tol, prec, 100000, nullptr, nullptr);
            if (s != WD_OK) return s;
            k_weight_g5<<<eb, 256, 0, c->st>>>(g, we, wo, we, wo, one_d, 1, nb);       // g5 (.)
            c->launches += 2;
        }
        WD_CUDA(cudaGetLastError());
        // link force, scaled by 1/N for the mean over samples
        WD_TRY(force_eo(c, we, wo, ze, zo, nb, scale, G, H, first ? 0 : 1));
        first = false;
        // kappa: sum_rhs (w^dag z - (B v)^dag z) / (kappa N)
        const long per = 12L * g.Vh;
        k_dot_eo<<<nb, 256, 0, c->st>>>(we, wo, ze, zo, per, nb, dots);
        k_dot_eo<<<nb, 256, 0, c->st>>>(se, so, ze, zo, per, nb, dots + 2 * nb);
        c->launches += 2;
        std::vector<double> h(4 * nb);
        WD_CUDA(cudaMemcpyAsync(h.data(), dots, sizeof(double) * 4 * nb, cudaMemcpyDeviceToHost, c->st));
        WD_CUDA(cudaStreamSynchronize(c->st));
        for (int r = 0; r < nb; ++r) dk_re += h[2 * r] - h[2 * nb + 2 * r];
    }
    *dkappa = dk_re * scale / c->kappa;
    WD_CUDA(cudaStreamSynchronize(c->st));
    return WD_OK;
}
