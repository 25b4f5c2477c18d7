// Third multigrid level and the three-level MLMC estimator (Sec. 2 with
// L = 3, Eqs. 7-12; the three-level hierarchy of the paper's Table 2).
//
// The coarse lattice (extents cd, coarse dof 2 nv X + nv h + k) is aggregated
// again by agg2 coarse sites per direction.  Level-2 test vectors are
// restricted to each (level-3 aggregate, chirality half h) and orthonormalised
// by modified Gram-Schmidt in test-vector order, giving P_2 (level-3 dof
// 2 nv2 Xcc + nv2 h + k); D_3 = P_2^dag D_c P_2 is again a 9-point block
// stencil.  A level-2 stencil entry (X, b') lands in block 0 of D_3 unless the
// hop crosses the boundary of X's level-3 aggregate in its direction, then in
// the block of that direction -- so coincident neighbours (level-3 extents 1
// or 2) are never counted twice.
//
//   tr(B D^{-1}) = tr(B M_1) + tr(B P_1 M_2 P_1^dag) + tr(B P_1 P_2 D_3^{-1} P_2^dag P_1^dag),
//   M_1 = D^{-1} - P_1 D_2^{-1} P_1^dag,   M_2 = D_2^{-1} - P_2 D_3^{-1} P_2^dag,
// level 1 on fine noise, level 2 on coarse noise xi (samples | 2^23), level 3
// on level-3 noise zeta (samples | 2^24).
#include <math.h>
#include <string.h>

#include <vector>

#include "wd_internal.h"

namespace wd {

struct Mg3Geom {
    int cd[4], agg2[4], cd3[4];
    int nv, ncd, nv2, ncd2, Vc, Vcc;
};

__device__ __forceinline__ void site_coords(int X, const int d[4], int c[4]) {
    for (int m = 0; m < 4; ++m) { c[m] = X % d[m]; X /= d[m]; }
}
__device__ __forceinline__ int site_index(const int c[4], const int d[4]) {
    return c[0] + d[0] * (c[1] + d[1] * (c[2] + d[2] * c[3]));
}
// level-2 site of the j-th member of level-3 aggregate Xcc
__device__ __forceinline__ int member(const Mg3Geom &M, int Xcc, int j) {
    int a[4], c[4];
    site_coords(Xcc, M.cd3, a);
    for (int m = 0; m < 4; ++m) { c[m] = a[m] * M.agg2[m] + j % M.agg2[m]; j /= M.agg2[m]; }
    return site_index(c, M.cd);
}
__device__ __forceinline__ int parent(const Mg3Geom &M, int X) {
    int c[4];
    site_coords(X, M.cd, c);
    for (int m = 0; m < 4; ++m) c[m] /= M.agg2[m];
    return site_index(c, M.cd3);
}

__device__ __forceinline__ double2 zmul_conj(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// test vectors [nv2][Vc][ncd] -> P2 [Vc][ncd][nv2]
__global__ void k_tv2_to_P2(const double2 *tv, double2 *P2, Mg3Geom M) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    const long n = (long)M.Vc * M.ncd * M.nv2;
    if (i >= n) return;
    const int k = (int)(i % M.nv2);
    const long xi = i / M.nv2;             // X * ncd + dof
    P2[i] = tv[(size_t)k * M.Vc * M.ncd + xi];
}

__device__ double2 block_sum_z(double2 v, double2 *sh) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double2 a = make_double2(0, 0);
    for (int w = 0; w < nw; ++w) { a.x += sh[w].x; a.y += sh[w].y; }
    return a;
}

// modified Gram-Schmidt of the nv2 columns of one (level-3 aggregate, half);
// rows: (member j, q < nv) -> coarse dof nv*h + q of member X_j; one CTA each
__global__ void k_block_mgs2(double2 *P2, Mg3Geom M) {
    __shared__ double2 sh[32];
    const int Xcc = blockIdx.x >> 1, h = blockIdx.x & 1;
    const int nmem = M.agg2[0] * M.agg2[1] * M.agg2[2] * M.agg2[3];
    const int m = nmem * M.nv;
    auto at = [&](int row, int k) -> double2 & {
        const int X = member(M, Xcc, row / M.nv), i = M.nv * h + row % M.nv;
        return P2[((size_t)X * M.ncd + i) * M.nv2 + k];
    };
    for (int k = 0; k < M.nv2; ++k) {
        for (int j = 0; j < k; ++j) {
            double2 d = make_double2(0, 0);
            for (int row = threadIdx.x; row < m; row += blockDim.x) {
                const double2 pj = at(row, j), pk = at(row, k);
                const double2 t = zmul_conj(pj, pk);
                d.x += t.x; d.y += t.y;
            }
            d = block_sum_z(d, sh);
            for (int row = threadIdx.x; row < m; row += blockDim.x) {
                double2 &q = at(row, k);
                const double2 qj = at(row, j);
                q.x -= d.x * qj.x - d.y * qj.y;
                q.y -= d.x * qj.y + d.y * qj.x;
            }
            __syncthreads();
        }
        double2 nn = make_double2(0, 0);
        for (int row = threadIdx.x; row < m; row += blockDim.x) {
            const double2 q = at(row, k);
            nn.x += q.x * q.x + q.y * q.y;
        }
        nn = block_sum_z(nn, sh);
        const double inv = 1.0 / sqrt(nn.x);
        for (int row = threadIdx.x; row < m; row += blockDim.x) {
            double2 &q = at(row, k);
            q.x *= inv;
            q.y *= inv;
        }
        __syncthreads();
    }
}

// level-3 neighbour table: b = 0 self, 1+mu forward, 5+mu backward
__global__ void k_nbr3(int *nbr, Mg3Geom M) {
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= M.Vcc) return;
    int c[4];
    site_coords(X, M.cd3, c);
    nbr[X * 9] = X;
    for (int mu = 0; mu < 4; ++mu)
        for (int dir = 0; dir < 2; ++dir) {
            int y[4] = {c[0], c[1], c[2], c[3]};
            y[mu] = dir == 0 ? (y[mu] + 1) % M.cd3[mu] : (y[mu] + M.cd3[mu] - 1) % M.cd3[mu];
            nbr[X * 9 + 1 + mu + 4 * dir] = site_index(y, M.cd3);
        }
}

// block of D_3 that level-2 stencil entry (X, b') contributes to
__device__ __forceinline__ int block3_of(const Mg3Geom &M, int X, int bp) {
    if (bp == 0) return 0;
    const int mu = (bp - 1) & 3;
    const bool fwd = bp <= 4;
    int c[4];
    site_coords(X, M.cd, c);
    const int r = c[mu] % M.agg2[mu];
    const bool crosses = fwd ? r == M.agg2[mu] - 1 : r == 0;
    return crosses ? bp : 0;
}

// D_3[Xcc][b] = sum over members X and level-2 entries b' that land in block b
// of P_2(X)^dag D_c[X][b'] P_2(nbr(X, b')).  One CTA per (Xcc, b); shared
// memory: the block (ncd2^2) and W = D_c[X][b'] P_2(Y) (ncd x ncd2).
__global__ void k_assemble3(const double2 *P2, const double2 *Dc, const int *nbr2, double2 *D3, Mg3Geom M) {
    extern __shared__ double2 sm[];
    double2 *A = sm, *W = sm + (size_t)M.ncd2 * M.ncd2;
    const int Xcc = blockIdx.x / 9, b = blockIdx.x % 9;
    const int n2 = M.ncd2 * M.ncd2, nw = M.ncd * M.ncd2;
    for (int e = threadIdx.x; e < n2; e += blockDim.x) A[e] = make_double2(0, 0);
    const int nmem = M.agg2[0] * M.agg2[1] * M.agg2[2] * M.agg2[3];
    for (int j = 0; j < nmem; ++j) {
        const int X = member(M, Xcc, j);
        for (int bp = 0; bp < 9; ++bp) {
            if (block3_of(M, X, bp) != b) continue;           // uniform over the CTA
            const int Y = nbr2[X * 9 + bp];
            const double2 *Db = Dc + ((size_t)X * 9 + bp) * M.ncd * M.ncd;
            __syncthreads();
            // W[i][c] = sum_{i' in half(c)} D_b[i][i'] P2[Y][i'][k(c)]
            for (int e = threadIdx.x; e < nw; e += blockDim.x) {
                const int i = e / M.ncd2, cc = e % M.ncd2, hc = cc / M.nv2, kc = cc % M.nv2;
                double2 acc = make_double2(0, 0);
                for (int q = 0; q < M.nv; ++q) {
                    const int ip = M.nv * hc + q;
                    const double2 d = Db[(size_t)i * M.ncd + ip], p = P2[((size_t)Y * M.ncd + ip) * M.nv2 + kc];
                    acc.x += d.x * p.x - d.y * p.y;
                    acc.y += d.x * p.y + d.y * p.x;
                }
                W[e] = acc;
            }
            __syncthreads();
            // A[a][c] += sum_{i in half(a)} conj(P2[X][i][k(a)]) W[i][c]
            for (int e = threadIdx.x; e < n2; e += blockDim.x) {
                const int a = e / M.ncd2, cc = e % M.ncd2, ha = a / M.nv2, ka = a % M.nv2;
                double2 acc = A[e];
                for (int q = 0; q < M.nv; ++q) {
                    const int i = M.nv * ha + q;
                    const double2 t = zmul_conj(P2[((size_t)X * M.ncd + i) * M.nv2 + ka], W[(size_t)i * M.ncd2 + cc]);
                    acc.x += t.x;
                    acc.y += t.y;
                }
                A[e] = acc;
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n2; e += blockDim.x) D3[((size_t)Xcc * 9 + b) * n2 + e] = A[e];
}

// y3[r][Xcc][nv2 h + k] = sum_{X in Xcc, q} conj(P2[X][nv h + q][k]) y2[r][X][nv h + q]
__global__ void k_restrict2(const double2 *P2, const double2 *y2, double2 *y3, Mg3Geom M, int nrhs) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)nrhs * M.Vcc * M.ncd2) return;
    const int a = (int)(t % M.ncd2);
    const long rest = t / M.ncd2;
    const int Xcc = (int)(rest % M.Vcc), r = (int)(rest / M.Vcc);
    const int h = a / M.nv2, k = a % M.nv2;
    const int nmem = M.agg2[0] * M.agg2[1] * M.agg2[2] * M.agg2[3];
    double2 acc = make_double2(0, 0);
    for (int j = 0; j < nmem; ++j) {
        const int X = member(M, Xcc, j);
        for (int q = 0; q < M.nv; ++q) {
            const int i = M.nv * h + q;
            const double2 tq = zmul_conj(P2[((size_t)X * M.ncd + i) * M.nv2 + k], y2[((size_t)r * M.Vc + X) * M.ncd + i]);
            acc.x += tq.x;
            acc.y += tq.y;
        }
    }
    y3[t] = acc;
}

// y2[r][X][i] = sum_k P2[X][i][k] y3[r][parent(X)][nv2 h(i) + k]  (overwrites y2)
__global__ void k_prolong2(const double2 *P2, const double2 *y3, double2 *y2, Mg3Geom M, int nrhs) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)nrhs * M.Vc * M.ncd) return;
    const int i = (int)(t % M.ncd);
    const long rest = t / M.ncd;
    const int X = (int)(rest % M.Vc), r = (int)(rest / M.Vc);
    const int h = i / M.nv, Xcc = parent(M, X);
    const double2 *yv = y3 + ((size_t)r * M.Vcc + Xcc) * M.ncd2 + (size_t)h * M.nv2;
    const double2 *pr = P2 + ((size_t)X * M.ncd + i) * M.nv2;
    double2 acc = make_double2(0, 0);
    for (int k = 0; k < M.nv2; ++k) {
        acc.x += pr[k].x * yv[k].x - pr[k].y * yv[k].y;
        acc.y += pr[k].x * yv[k].y + pr[k].y * yv[k].x;
    }
    y2[t] = acc;
}

// level-3 Rademacher noise: samples (sample0 + r) | 2^24 over the level-3 dofs
__global__ void k_noise3(double2 *z, unsigned long long seed, int sample0, long n3, int nrhs) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= n3 * nrhs) return;
    const unsigned long long r = (unsigned long long)(i / n3), j = (unsigned long long)(i % n3);
    const unsigned long long sample = ((unsigned long long)sample0 + r) | (1ULL << 24);
    unsigned long long h = seed ^ (sample << 40) ^ j;
    h += 0x9E3779B97F4A7C15ULL;
    h = (h ^ (h >> 30)) * 0xBF58476D1CE4E5B9ULL;
    h = (h ^ (h >> 27)) * 0x94D049BB133111EBULL;
    h ^= h >> 31;
    z[i] = make_double2((h >> 63) ? -1.0 : 1.0, 0.0);
}

__global__ void k_sub3(double2 *z, const double2 *w, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        z[i].x -= w[i].x;
        z[i].y -= w[i].y;
    }
}

}  // namespace wd

namespace wd {

int block_stencil_apply64(wd_ctx *c, const double2 *A, const int *nbr, int n, int V, const double *x, double *y,
                          const double *w, double a, double beta, int nrhs);   // wd_mg.cu
int coarse_solve(wd_ctx *c, const double *b, double *x, int nrhs, double tol, int prec, int max_iter,
                 double *resid_out);
int gen_noise_eo(wd_ctx *c, uint64_t seed, int sample0, int nrhs, double *be, double *bo);
int contract_noise_eo(wd_ctx *c, uint64_t seed, int sample0, int nrhs, int gamma5, const double *ye,
                      const double *yo, double *X);
int auto_batch(wd_ctx *c, int total);
int mlmc_contract_fields(wd_ctx *c, const double *ae, const double *ao, const double *be, const double *bo,
                         int gamma5, int nrhs, double *X, int sample0);              // wd_mlmc.cu
int mlmc_mean_var(wd_ctx *c, const double *X, int N, double *mean, double *var);     // wd_mlmc.cu
int coarse_noise_dev(wd_ctx *c, double *xi, uint64_t seed, int sample0, long ncoarse, int nrhs);   // wd_mlmc.cu
int mlmc_combine3(wd_ctx *c, const double *m1, const double *v1, const double *m2, const double *v2,
                  const double *m3, const double *v3, int N1, int N2, int N3, double *mean, double *var);

static Mg3Geom mg3_geom(wd_ctx *c) {
    Mg3Geom M;
    for (int m = 0; m < 4; ++m) { M.cd[m] = c->mg->cd[m]; M.agg2[m] = c->mg3->agg2[m]; M.cd3[m] = c->mg3->cd3[m]; }
    M.nv = c->mg->nv; M.ncd = c->mg->ncd; M.Vc = c->mg->Vc;
    M.nv2 = c->mg3->nv2; M.ncd2 = c->mg3->ncd2; M.Vcc = c->mg3->Vcc;
    return M;
}

static Space level3_space(wd_ctx *c) {
    Space s;
    s.units = (long)c->mg3->Vcc * c->mg3->ncd2 / 12;
    s.flat = true;
    return s;
}

int apply3(wd_ctx *c, const double *x, double *y, const double *w, double a, double beta, int nrhs) {
    return block_stencil_apply64(c, c->mg3->D3, c->mg3->nbr3, c->mg3->ncd2, c->mg3->Vcc, x, y, w, a, beta, nrhs);
}
static int op3(wd_ctx *c, const void *in, void *out, int nrhs, void *) {
    return apply3(c, (const double *)in, (double *)out, nullptr, 0.0, 1.0, nrhs);
}
static int res3(wd_ctx *c, const double *b, const double *x, double *r, int nrhs, void *) {
    return apply3(c, x, r, b, 1.0, -1.0, nrhs);
}

int restrict2(wd_ctx *c, const double *y2, double *y3, int nrhs) {
    const Mg3Geom M = mg3_geom(c);
    const long n = (long)nrhs * M.Vcc * M.ncd2;
    k_restrict2<<<(unsigned)((n + 127) / 128), 128, 0, c->st>>>(c->mg3->P2, (const double2 *)y2, (double2 *)y3, M,
                                                                 nrhs);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int prolong2(wd_ctx *c, const double *y3, double *y2, int nrhs) {
    const Mg3Geom M = mg3_geom(c);
    const long n = (long)nrhs * M.Vc * M.ncd;
    k_prolong2<<<(unsigned)((n + 127) / 128), 128, 0, c->st>>>(c->mg3->P2, (const double2 *)y3, (double2 *)y2, M,
                                                                nrhs);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// x = D_3^{-1} b (FP64 BiCGStab on the level-3 vectors [nrhs][Vcc][ncd2])
int solve3(wd_ctx *c, const double *b, double *x, int nrhs, double tol, int max_iter) {
    const Space sp = level3_space(c);
    double *bn2;
    WD_TRY(ws_get(c, "l3.bn2", sizeof(double) * nrhs, (void **)&bn2));
    WD_TRY(blas_norm2(c, sp, P64, b, nrhs, bn2));
    std::vector<double> bnorm2(nrhs);
    WD_CUDA(cudaMemcpyAsync(bnorm2.data(), bn2, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaStreamSynchronize(c->st));
    Problem P;
    P.sp = sp;
    P.op64 = op3; P.u64 = nullptr;
    P.oplo = op3; P.ulo = nullptr;
    P.res64 = res3; P.ures = nullptr;
    P.tag = "level3";
    std::vector<int> iters;
    std::vector<double> last;
    return dc_solve(c, P, b, x, nrhs, bn2, bnorm2, tol, P64, max_iter, iters, last);
}

}  // namespace wd

using namespace wd;

void wd_mg3_free(wd_ctx *c) {
    if (!c || !c->mg3) return;
    cudaStreamSynchronize(c->st);
    wd_mg3 *g = c->mg3;
    if (g->P2) cudaFree(g->P2);
    if (g->D3) cudaFree(g->D3);
    if (g->nbr3) cudaFree(g->nbr3);
    delete g;
    c->mg3 = nullptr;
}

extern "C" int wd_mg3_setup(wd_ctx *c, const double *tv2, int nv2, const int agg2[4], int tv_iters, uint64_t seed) {
    if (!c || !agg2 || nv2 < 1 || nv2 % 6 != 0 || tv_iters < 0) {
        set_error("wd_mg3_setup: bad argument (nv2 must be a positive multiple of 6)");
        return WD_EINVAL;
    }
    if (!c->mg) { set_error("wd_mg3_setup: needs wd_mg_setup first"); return WD_EINVAL; }
    int nmem = 1;
    for (int m = 0; m < 4; ++m) {
        if (agg2[m] < 1 || c->mg->cd[m] % agg2[m]) {
            set_error("wd_mg3_setup: aggregate extent %d does not divide the coarse extent %d", agg2[m], c->mg->cd[m]);
            return WD_EINVAL;
        }
        nmem *= agg2[m];
    }
    const int nv = c->mg->nv, ncd = c->mg->ncd, ncd2 = 2 * nv2;
    if (nv2 > nv * nmem) { set_error("wd_mg3_setup: nv2 > nv * aggregate volume"); return WD_EINVAL; }
    const size_t smem = sizeof(double2) * ((size_t)ncd2 * ncd2 + (size_t)ncd * ncd2);
    if (smem > 227 * 1024) { set_error("wd_mg3_setup: nv2 too large for the block assembly"); return WD_ENOTSUP; }
    wd_mg3_free(c);
    wd_mg3 *g = new wd_mg3();
    memset(g, 0, sizeof(*g));
    c->mg3 = g;
    g->nv2 = nv2;
    g->ncd2 = ncd2;
    g->Vcc = 1;
    for (int m = 0; m < 4; ++m) { g->agg2[m] = agg2[m]; g->cd3[m] = c->mg->cd[m] / agg2[m]; g->Vcc *= g->cd3[m]; }
    const long n2 = (long)c->mg->Vc * ncd;
    const size_t nP = (size_t)n2 * nv2, nD = (size_t)g->Vcc * 9 * ncd2 * ncd2;
    if (cudaMalloc(&g->P2, nP * sizeof(double2)) != cudaSuccess || cudaMalloc(&g->D3, nD * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&g->nbr3, sizeof(int) * 9 * g->Vcc) != cudaSuccess) {
        cudaGetLastError();
        wd_mg3_free(c);
        set_error("wd_mg3_setup: allocation failed");
        return WD_ENOMEM;
    }
    double *tvd;
    WD_TRY(ws_get(c, "mg3.tv", nP * sizeof(double2), (void **)&tvd));
    if (tv2) {
        WD_CUDA(cudaMemcpyAsync(tvd, tv2, nP * sizeof(double2), cudaMemcpyHostToDevice, c->st));
    } else {
        // inverse iterations on level 2: random coarse vectors, v <- D_2^{-1} v / |.|
        double *tmp, *nrm;
        WD_TRY(ws_get(c, "mg3.tmp", nP * sizeof(double2), (void **)&tmp));
        WD_TRY(ws_get(c, "mg3.nrm", sizeof(double) * nv2, (void **)&nrm));
        WD_TRY(coarse_noise_dev(c, tvd, seed, 1 << 22, n2, nv2));
        for (int it = 0; it < tv_iters; ++it) {
            int s = coarse_solve(c, tvd, tmp, nv2, 1e-6, P32, 100000, nullptr);
            if (s != WD_OK && s != WD_ENOCONV) return s;
            WD_CUDA(cudaMemcpyAsync(tvd, tmp, nP * sizeof(double2), cudaMemcpyDeviceToDevice, c->st));
        }
    }
    const Mg3Geom M = mg3_geom(c);
    k_tv2_to_P2<<<(unsigned)((nP + 255) / 256), 256, 0, c->st>>>((const double2 *)tvd, g->P2, M);
    k_block_mgs2<<<2 * g->Vcc, 256, 0, c->st>>>(g->P2, M);
    k_nbr3<<<(g->Vcc + 127) / 128, 128, 0, c->st>>>(g->nbr3, M);
    WD_CUDA(cudaFuncSetAttribute(k_assemble3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_assemble3<<<9 * g->Vcc, 256, smem, c->st>>>(g->P2, c->mg->Dc, c->mg->nbr, g->D3, M);
    c->launches += 4;
    WD_CUDA(cudaGetLastError());
    WD_CUDA(cudaStreamSynchronize(c->st));
    return WD_OK;
}

// y = D_3 x on level-3 vectors [nrhs][Vcc][2 nv2] (device complex128)
extern "C" int wd_coarse3_apply(wd_ctx *c, const double *in, double *out, int nrhs) {
    if (!c || !c->mg3 || nrhs < 0 || ((!in || !out) && nrhs > 0)) { set_error("wd_coarse3_apply: bad argument or no third level"); return WD_EINVAL; }
    if (nrhs == 0) return WD_OK;
    WD_TRY(apply3(c, in, out, nullptr, 0.0, 1.0, nrhs));
    WD_CUDA(cudaStreamSynchronize(c->st));
    return WD_OK;
}

// level-2 <-> level-3 transfer (device complex128): y3 = P_2^dag y2, y2 = P_2 y3
extern "C" int wd_restrict2(wd_ctx *c, const double *y2, double *y3, int nrhs) {
    if (!c || !c->mg3 || nrhs < 0) { set_error("wd_restrict2: bad argument or no third level"); return WD_EINVAL; }
    if (nrhs == 0) return WD_OK;
    WD_TRY(restrict2(c, y2, y3, nrhs));
    WD_CUDA(cudaStreamSynchronize(c->st));
    return WD_OK;
}
extern "C" int wd_prolong2(wd_ctx *c, const double *y3, double *y2, int nrhs) {
    if (!c || !c->mg3 || nrhs < 0) { set_error("wd_prolong2: bad argument or no third level"); return WD_EINVAL; }
    if (nrhs == 0) return WD_OK;
    WD_TRY(prolong2(c, y3, y2, nrhs));
    WD_CUDA(cudaStreamSynchronize(c->st));
    return WD_OK;
}

// Three-level MLMC estimate of tr[B D^{-1}(t, t)] (Eq. 12 with L = 3).
extern "C" int trace_estimate_mlmc3(wd_ctx *c, int N1, int N2, int N3, uint64_t seed, int op, int prec, int batch,
                                    double tol, double *estimate, double *sample_var, int64_t *n_solves_out,
                                    double *samples1, double *samples2, double *samples3) {
    if (!c || !estimate || !sample_var || N1 < 2 || N2 < 2 || N3 < 2 || prec < 0 || prec > 2 || !(tol > 0) ||
        (op != 0 && op != 1)) {
        set_error("trace_estimate_mlmc3: bad argument (N1, N2, N3 >= 2)");
        return WD_EINVAL;
    }
    if (!c->mg || !c->mg3) { set_error("trace_estimate_mlmc3: needs wd_mg_setup and wd_mg3_setup"); return WD_EINVAL; }
    const Geom &g = c->g;
    const int T = g.T;
    const long n2 = (long)c->mg->Vc * c->mg->ncd, n3 = (long)c->mg3->Vcc * c->mg3->ncd2;
    double *X[3];
    const int Ns[3] = {N1, N2, N3};
    for (int l = 0; l < 3; ++l) {
        char name[16];
        snprintf(name, sizeof(name), "ml3.X%d", l);
        WD_TRY(ws_get(c, name, sizeof(double) * 2 * (size_t)Ns[l] * T, (void **)&X[l]));
        WD_CUDA(cudaMemsetAsync(X[l], 0, sizeof(double) * 2 * (size_t)Ns[l] * T, c->st));
    }
    int64_t ns = 0;
    const int Nmax = N1 > N2 ? (N1 > N3 ? N1 : N3) : (N2 > N3 ? N2 : N3);
    const int B = batch > 0 ? batch : auto_batch(c, Nmax);
    const double l3tol = tol < 1e-12 ? tol : 1e-12;     // level 3 is tiny: solve it tightly in FP64
    for (int level = 1; level <= 3; ++level) {
        const int N = Ns[level - 1];
        for (int s0 = 0; s0 < N; s0 += B) {
            const int nb = N - s0 < B ? N - s0 : B;
            const size_t f = field_bytes(g, P64, nb);
            double *ae, *ao, *be, *bo, *c2a, *c2b, *c3a, *c3b;
            WD_TRY(ws_get(c, "ml3.ae", f, (void **)&ae));
            WD_TRY(ws_get(c, "ml3.ao", f, (void **)&ao));
            WD_TRY(ws_get(c, "ml3.be", f, (void **)&be));
            WD_TRY(ws_get(c, "ml3.bo", f, (void **)&bo));
            WD_TRY(ws_get(c, "ml3.c2a", sizeof(double2) * n2 * nb, (void **)&c2a));
            WD_TRY(ws_get(c, "ml3.c2b", sizeof(double2) * n2 * nb, (void **)&c2b));
            WD_TRY(ws_get(c, "ml3.c3a", sizeof(double2) * n3 * nb, (void **)&c3a));
            WD_TRY(ws_get(c, "ml3.c3b", sizeof(double2) * n3 * nb, (void **)&c3b));
            int s;
            if (level == 1) {
                // eta^dag B (D^{-1} eta - P_1 D_2^{-1} P_1^dag eta)
                WD_TRY(gen_noise_eo(c, seed, s0, nb, ae, ao));
                s = solve_eo(c, ae, ao, be, bo, nb, tol, prec, 100000, nullptr, nullptr);
                if (s != WD_OK) return s;
                WD_TRY(mg_restrict_eo(c, ae, ao, c2a, nb, true));
                s = coarse_solve(c, c2a, c2b, nb, tol, prec, 100000, nullptr);
                if (s != WD_OK) return s;
                double *we, *wo;
                WD_TRY(ws_get(c, "ml3.we", f, (void **)&we));
                WD_TRY(ws_get(c, "ml3.wo", f, (void **)&wo));
                WD_TRY(mg_prolong_eo(c, c2b, we, wo, nb, true));
                const long nf = (long)nb * 24 * g.Vh;
                k_sub3<<<1184, 256, 0, c->st>>>((double2 *)be, (const double2 *)we, nf / 2);
                k_sub3<<<1184, 256, 0, c->st>>>((double2 *)bo, (const double2 *)wo, nf / 2);
                c->launches += 2;
                WD_TRY(contract_noise_eo(c, seed, s0, nb, op, be, bo, X[0]));
                ns += 2 * nb;
            } else if (level == 2) {
                // (P_1 xi)^dag B P_1 (D_2^{-1} xi - P_2 D_3^{-1} P_2^dag xi)
                WD_TRY(coarse_noise_dev(c, c2a, seed, s0, n2, nb));
                s = coarse_solve(c, c2a, c2b, nb, tol, prec, 100000, nullptr);
                if (s != WD_OK) return s;
                WD_TRY(restrict2(c, c2a, c3a, nb));
                s = solve3(c, c3a, c3b, nb, l3tol, 100000);
                if (s != WD_OK) return s;
                double *c2w;
                WD_TRY(ws_get(c, "ml3.c2w", sizeof(double2) * n2 * nb, (void **)&c2w));
                WD_TRY(prolong2(c, c3b, c2w, nb));
                k_sub3<<<1184, 256, 0, c->st>>>((double2 *)c2b, (const double2 *)c2w, n2 * nb);
                c->launches++;
                WD_TRY(mg_prolong_eo(c, c2a, ae, ao, nb, true));
                WD_TRY(mg_prolong_eo(c, c2b, be, bo, nb, true));
                WD_TRY(mlmc_contract_fields(c, ae, ao, be, bo, op, nb, X[1], s0));
                ns += 2 * nb;
            } else {
                // (P_1 P_2 zeta)^dag B (P_1 P_2 D_3^{-1} zeta)
                const long n = n3 * nb;
                k_noise3<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>((double2 *)c3a, seed, s0, n3, nb);
                c->launches++;
                s = solve3(c, c3a, c3b, nb, l3tol, 100000);
                if (s != WD_OK) return s;
                WD_TRY(prolong2(c, c3a, c2a, nb));
                WD_TRY(prolong2(c, c3b, c2b, nb));
                WD_TRY(mg_prolong_eo(c, c2a, ae, ao, nb, true));
                WD_TRY(mg_prolong_eo(c, c2b, be, bo, nb, true));
                WD_TRY(mlmc_contract_fields(c, ae, ao, be, bo, op, nb, X[2], s0));
                ns += nb;
            }
        }
    }
    double *mv[6], *mean, *var;
    for (int k = 0; k < 6; ++k) {
        char name[16];
        snprintf(name, sizeof(name), "ml3.mv%d", k);
        WD_TRY(ws_get(c, name, sizeof(double) * 2 * (T + 1), (void **)&mv[k]));
    }
    WD_TRY(ws_get(c, "ml3.mean", sizeof(double) * 2 * (T + 1), (void **)&mean));
    WD_TRY(ws_get(c, "ml3.var", sizeof(double) * (T + 1), (void **)&var));
    for (int l = 0; l < 3; ++l) WD_TRY(mlmc_mean_var(c, X[l], Ns[l], mv[2 * l], mv[2 * l + 1]));
    WD_TRY(mlmc_combine3(c, mv[0], mv[1], mv[2], mv[3], mv[4], mv[5], N1, N2, N3, mean, var));
    WD_CUDA(cudaMemcpyAsync(estimate, mean, sizeof(double) * 2 * (T + 1), cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaMemcpyAsync(sample_var, var, sizeof(double) * (T + 1), cudaMemcpyDeviceToHost, c->st));
    double *outs[3] = {samples1, samples2, samples3};
    for (int l = 0; l < 3; ++l)
        if (outs[l])
            WD_CUDA(cudaMemcpyAsync(outs[l], X[l], sizeof(double) * 2 * (size_t)Ns[l] * T, cudaMemcpyDeviceToHost,
                                    c->st));
    WD_CUDA(cudaStreamSynchronize(c->st));
    WD_TRY(hop_err_check(c));
    if (n_solves_out) *n_solves_out = ns;
    return WD_OK;
}
