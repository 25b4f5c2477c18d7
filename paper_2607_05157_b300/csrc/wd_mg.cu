// Two-level aggregation multigrid for the MLMC estimator (Sec. 2).
//
// Transfer operators (Sec. 2: R = P^dag, P^dag P = I): the fine lattice is cut
// into aggregates of agg[mu] sites per direction; every test vector is
// restricted to each aggregate and each chirality half (g5 = +1: spins 0, 1;
// g5 = -1: spins 2, 3) and the restricted vectors of one (aggregate, half)
// are orthonormalised by modified Gram-Schmidt in test-vector order.  Coarse
// dof i = nv*h + k of coarse site X (ncd = 2 nv dofs per site).
// P is stored per fine site: P[parity][s][12][nv] complex (eo site order),
// entry [x][3*spin+colour][k] = component of column (X(x), half(spin), k).
//
// Galerkin operator (Eq. 7): D_c = P^dag D P.  Because D couples nearest
// neighbours and P is block diagonal over aggregates, D_c is a 9-point
// stencil of ncd x ncd blocks:
//   y(X) = A_0(X) x(X) + sum_mu [A_{+mu}(X) x(X+mu) + A_{-mu}(X) x(X-mu)],
// A_0 collecting the identity and every hop that stays inside X, A_{+-mu}
// the hops that leave X through its +-mu face (with a coarse extent of 1 or
// 2 the neighbour is X itself or the same site twice; the blocks stay
// separate and their contributions add).  The blocks are assembled directly
// from the links and P, hop by hop, in FP64.
#include <math.h>
#include <string.h>

#include <vector>

#include <chrono>

#include "wd_internal.h"
#include "wd_dd.cuh"



namespace wd {

// g_mu in the chiral basis: g_k = [[0, -i s_k], [i s_k, 0]], g_4 = [[0, 1], [1, 0]]
__constant__ double2 c_gamma[4][4][4];

static void host_gamma(double2 g[4][4][4]) {
    memset(g, 0, sizeof(double2) * 64);
    // sigma matrices (re, im)
    const double s[3][2][2][2] = {{{{0, 0}, {1, 0}}, {{1, 0}, {0, 0}}},
                                  {{{0, 0}, {0, -1}}, {{0, 1}, {0, 0}}},
                                  {{{1, 0}, {0, 0}}, {{0, 0}, {-1, 0}}}};
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const double re = s[k][a][b][0], im = s[k][a][b][1];
                // upper right: -i s = (im, -re);  lower left: i s = (-im, re)
                g[k][a][2 + b] = make_double2(im, -re);
                g[k][2 + a][b] = make_double2(-im, re);
            }
    for (int a = 0; a < 2; ++a) { g[3][a][2 + a] = make_double2(1, 0); g[3][2 + a][a] = make_double2(1, 0); }
}

__device__ __forceinline__ double2 zfma(double2 acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
__device__ __forceinline__ double2 zfma_conj(double2 acc, double2 a, double2 b) {   // acc += conj(a) b
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}

struct MgGeom {
    Geom g;
    int agg[4], cd[4];
    int nv, ncd, Vc;
};

// fine site (lexicographic) of the j-th site of aggregate X, j in [0, prod agg)
__device__ __forceinline__ void agg_site(const MgGeom &M, int X, int j, int c[4]) {
    int xc[4];
    int r = X;
    for (int m = 0; m < 4; ++m) { xc[m] = r % M.cd[m]; r /= M.cd[m]; }
    int q = j;
    for (int m = 0; m < 4; ++m) { c[m] = xc[m] * M.agg[m] + q % M.agg[m]; q /= M.agg[m]; }
}
__device__ __forceinline__ int lex(const Geom &g, const int c[4]) { return c[0] + g.X * (c[1] + g.Y * (c[2] + g.Z * c[3])); }
__device__ __forceinline__ int coarse_of(const MgGeom &M, const int c[4]) {
    return c[0] / M.agg[0] + M.cd[0] * (c[1] / M.agg[1] + M.cd[1] * (c[2] / M.agg[2] + M.cd[2] * (c[3] / M.agg[3])));
}
// P entry for (fine lexicographic site, component, k)
__device__ __forceinline__ size_t pidx(const MgGeom &M, int site, int comp, int k) {
    const int c0 = site % M.g.X, r = site / M.g.X;
    const int c1 = r % M.g.Y, c2 = (r / M.g.Y) % M.g.Z, c3 = r / (M.g.Y * M.g.Z);
    const int par = (c0 + c1 + c2 + c3) & 1;
    return (((size_t)par * M.g.Vh + (site >> 1)) * 12 + comp) * M.nv + k;
}

// test vectors (user layout [nv][V][12]) -> P layout
__global__ void k_tv_to_P(const double2 *tv, double2 *P, MgGeom M) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)M.g.V * 12 * M.nv) return;
    const int k = (int)(i % M.nv);
    const long rest = i / M.nv;
    const int comp = (int)(rest % 12), site = (int)(rest / 12);
    P[pidx(M, site, comp, k)] = tv[((size_t)k * M.g.V + site) * 12 + comp];
}

__device__ double2 block_reduce_z(double2 v, double2 *sh) {
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

// Column-major copy of the (aggregate, half) blocks of P for the block MGS:
// Pt[blk][k][row], blk = 2 X + h, row = 6 (site in aggregate) + (comp - 6 h),
// so that every MGS pass reads whole columns with coalesced loads.  One
// thread per (blk, row) moves the row's nv contiguous entries.
__global__ void k_mgs_gather(const double2 *P, double2 *Pt, MgGeom M, int to_blocks) {
    const int nsite = M.agg[0] * M.agg[1] * M.agg[2] * M.agg[3], m = nsite * 6;
    const long n = 2L * M.Vc * m;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
        const int row = (int)(t % m);
        const long blk = t / m;
        const int X = (int)(blk >> 1), h = (int)(blk & 1);
        int c[4];
        agg_site(M, X, row / 6, c);
        const size_t off = pidx(M, lex(M.g, c), 6 * h + row % 6, 0);
        double2 *col = Pt + (size_t)blk * M.nv * m + row;
        if (to_blocks)
            for (int k = 0; k < M.nv; ++k) col[(size_t)k * m] = P[off + k];
        else
            for (int k = 0; k < M.nv; ++k) ((double2 *)P)[off + k] = col[(size_t)k * m];
    }
}

// Modified Gram-Schmidt of the nv columns of one (aggregate, half) block of
// the column-major copy; one CTA per block.  Each pass over the rows
// subtracts q_j from v_k and, in the same pass, accumulates the next dot
// product q_{j+1}^dag v_k (or, after the last j, |v_k|^2) from the updated
// rows: the arithmetic of sequential MGS in its order, with half the passes.
__global__ void k_block_mgs_cm(double2 *Pt, MgGeom M) {
    __shared__ double2 sh[32];
    const int nsite = M.agg[0] * M.agg[1] * M.agg[2] * M.agg[3];
    const int m = nsite * 6;
    double2 *B = Pt + (size_t)blockIdx.x * M.nv * m;
    for (int k = 0; k < M.nv; ++k) {
        double2 *vk = B + (size_t)k * m;
        double2 d = make_double2(0, 0);
        if (k > 0) {
            for (int row = threadIdx.x; row < m; row += blockDim.x) d = zfma_conj(d, B[row], vk[row]);
            d = block_reduce_z(d, sh);
        }
        double2 nn = make_double2(0, 0);
        for (int j = 0; j < k; ++j) {
            const double2 *qj = B + (size_t)j * m, *qn = qj + m;
            double2 dn = make_double2(0, 0);
            for (int row = threadIdx.x; row < m; row += blockDim.x) {
                double2 q = vk[row];
                const double2 a = qj[row];
                q.x -= d.x * a.x - d.y * a.y;
                q.y -= d.x * a.y + d.y * a.x;
                vk[row] = q;
                if (j + 1 < k) dn = zfma_conj(dn, qn[row], q);
                else dn.x += q.x * q.x + q.y * q.y;
            }
            if (j + 1 < k) d = block_reduce_z(dn, sh);
            else nn = dn;
        }
        if (k == 0)
            for (int row = threadIdx.x; row < m; row += blockDim.x) {
                const double2 q = vk[row];
                nn.x += q.x * q.x + q.y * q.y;
            }
        nn = block_reduce_z(nn, sh);
        const double inv = 1.0 / sqrt(nn.x);
        for (int row = threadIdx.x; row < m; row += blockDim.x) {
            vk[row].x *= inv;
            vk[row].y *= inv;
        }
        __syncthreads();
    }
}

// The same MGS with one warp per block and four blocks per CTA: the column
// being orthogonalised lives in shared memory (m rows of 16 bytes per warp;
// lane l owns rows l, l + 32, ..., so no other lane touches them), the dot
// products reduce by warp shuffles, and no pass waits at a CTA barrier.
// Each pass subtracts q_j and accumulates the next dot product (or the norm)
// from the updated rows, as above.  On the 24^3x48 setup (5184 blocks of
// 1536 rows x 24 columns) it takes 55 ms against 72 ms for the CTA kernel;
// its ~24 G FP64 operations bound it near 40 ms at the FP64 rate.
__device__ __forceinline__ double2 warp_sum_z(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
__global__ void __launch_bounds__(128) k_block_mgs_warp(double2 *Pt, MgGeom M, int nblocks) {
    extern __shared__ double2 mgs_sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int blk = blockIdx.x * 4 + warp;
    if (blk >= nblocks) return;                            // uniform in the warp; no CTA barrier follows
    const int m = M.agg[0] * M.agg[1] * M.agg[2] * M.agg[3] * 6;
    double2 *vs = mgs_sm + (size_t)warp * m;
    double2 *B = Pt + (size_t)blk * M.nv * m;
    for (int k = 0; k < M.nv; ++k) {
        const double2 *vk = B + (size_t)k * m;
        for (int row = lane; row < m; row += 32) vs[row] = vk[row];
        double2 d = make_double2(0, 0), nn = make_double2(0, 0);
        if (k > 0) {
            double2 p = make_double2(0, 0);
            for (int row = lane; row < m; row += 32) p = zfma_conj(p, B[row], vs[row]);
            d = warp_sum_z(p);
        }
        for (int j = 0; j < k; ++j) {
            const double2 *qj = B + (size_t)j * m, *qn = qj + m;
            double2 dn = make_double2(0, 0);
            for (int row = lane; row < m; row += 32) {
                double2 q = vs[row];
                const double2 a = qj[row];
                q.x -= d.x * a.x - d.y * a.y;
                q.y -= d.x * a.y + d.y * a.x;
                vs[row] = q;
                if (j + 1 < k) dn = zfma_conj(dn, qn[row], q);
                else dn.x += q.x * q.x + q.y * q.y;
            }
            if (j + 1 < k) d = warp_sum_z(dn);
            else nn = dn;
        }
        if (k == 0)
            for (int row = lane; row < m; row += 32) {
                const double2 q = vs[row];
                nn.x += q.x * q.x + q.y * q.y;
            }
        nn = warp_sum_z(nn);
        const double inv = 1.0 / sqrt(nn.x);
        double2 *out = B + (size_t)k * m;
        for (int row = lane; row < m; row += 32) {
            const double2 q = vs[row];
            out[row] = make_double2(q.x * inv, q.y * inv);
        }
    }
}

// Gram matrices of P's columns restricted to one timeslice of an aggregate
// and one chirality half: Gt[X][tau][h][k][l] = sum over the sites x of
// aggregate X with t(x) = t0(X) + tau and the 6 components of half h of
// conj(P_k(x)) P_l(x).  Since P is block diagonal over aggregates and halves,
// sum_{x in t} (P a)(x)^dag B (P b)(x) = sum_{X, h} s_h a_{X,h}^dag Gt[X][t - t0(X)][h] b_{X,h}
// (s_h = +1, or +1 / -1 on the halves for B = g5): the per-timeslice trace
// contraction (Eq. 21) of two coarse vectors needs no fine fields.  One CTA
// per (X, tau, h).
__global__ void k_gram_t(const double2 *P, double2 *Gt, MgGeom M) {
    const int at = M.agg[3], nv = M.nv;
    const int b = blockIdx.x;                        // (X * at + tau) * 2 + h
    const int h = b & 1, tau = (b >> 1) % at, X = (b >> 1) / at;
    const int ns3 = M.agg[0] * M.agg[1] * M.agg[2];
    for (int e = threadIdx.x; e < nv * nv; e += blockDim.x) {
        const int k = e / nv, l = e % nv;
        double2 acc = make_double2(0, 0);
        for (int j3 = 0; j3 < ns3; ++j3) {
            int c[4];
            agg_site(M, X, j3 + ns3 * tau, c);       // time offset tau inside the aggregate
            const int site = lex(M.g, c);
            for (int r = 0; r < 6; ++r) {
                const int comp = 6 * h + r;
                acc = zfma_conj(acc, P[pidx(M, site, comp, k)], P[pidx(M, site, comp, l)]);
            }
        }
        Gt[(size_t)b * nv * nv + e] = acc;
    }
}

// The same Gram matrices in double-float arithmetic from the FP32 pair copy of
// P (Ph + Pl), the sites of the aggregate timeslice walked with an incremental
// counter (the FP64 rate is a small fraction of the FP32 one)
__global__ void k_gram_t_dd(const float2 *Ph, const float2 *Pl, double2 *Gt, MgGeom M) {
    const int at = M.agg[3], nv = M.nv;
    const int b = blockIdx.x;                        // (X * at + tau) * 2 + h
    const int h = b & 1, tau = (b >> 1) % at, X = (b >> 1) / at;
    int o[4];
    {
        int r = X;
        for (int m = 0; m < 4; ++m) { o[m] = (r % M.cd[m]) * M.agg[m]; r /= M.cd[m]; }
        o[3] += tau;
    }
    // G is hermitian: the entries k <= l, each written to (k, l) and its
    // conjugate to (l, k)
    const int npair = nv * (nv + 1) / 2;
    for (int e = threadIdx.x; e < npair; e += blockDim.x) {
        int k = 0, rem = e;
        while (rem >= nv - k) { rem -= nv - k; ++k; }
        const int l = k + rem;
        dd are = dd_make(0.f, 0.f), aim = dd_make(0.f, 0.f);
        for (int dz = 0; dz < M.agg[2]; ++dz)
            for (int dy = 0; dy < M.agg[1]; ++dy)
                for (int dx = 0; dx < M.agg[0]; ++dx) {
                    const int c0 = o[0] + dx, c1 = o[1] + dy, c2 = o[2] + dz;
                    const int site = c0 + M.g.X * (c1 + M.g.Y * (c2 + M.g.Z * o[3]));
                    const int par = (c0 + c1 + c2 + o[3]) & 1;
                    const size_t row = ((size_t)par * M.g.Vh + (site >> 1)) * 12 + 6 * h;
                    for (int r = 0; r < 6; ++r) {
                        const size_t qk = (row + r) * nv + k, ql = (row + r) * nv + l;
                        const float2 kh = __ldg(Ph + qk), kl = __ldg(Pl + qk), lh = __ldg(Ph + ql), ll = __ldg(Pl + ql);
                        const dd kr = dd_make(kh.x, kl.x), ki = dd_make(kh.y, kl.y);
                        const dd lr = dd_make(lh.x, ll.x), li = dd_make(lh.y, ll.y);
                        dd_fma(are, kr, lr);   // conj(P_k) P_l
                        dd_fma(are, ki, li);
                        dd_fma(aim, kr, li);
                        dd_fma(aim, -ki, lr);
                    }
                }
        const double gr = dd2d(are), gi = dd2d(aim);
        Gt[(size_t)b * nv * nv + (size_t)k * nv + l] = make_double2(gr, gi);
        if (l != k) Gt[(size_t)b * nv * nv + (size_t)l * nv + k] = make_double2(gr, -gi);
    }
}

// part[r][t] = sum_{X in timeslice t / agg_t} sum_h s_h a_{X,h}^dag Gt[X][t % agg_t][h] b_{X,h}
// for coarse vectors a, b [nrhs][Vc][2 nv]; one CTA per (r, t), a fixed
// assignment of (X, h, k) to threads and a fixed reduction order
__global__ void __launch_bounds__(256) k_contract_coarse_t(const double2 *Gt, const double2 *a, const double2 *b,
                                                           int gamma5, double *part, MgGeom M) {
    __shared__ double2 sh[32];
    const int r = blockIdx.x, t = blockIdx.y, T = M.g.T;
    const int at = M.agg[3], nv = M.nv, ncd = M.ncd;
    const int Vs = M.cd[0] * M.cd[1] * M.cd[2];
    const int ct = t / at, tau = t % at;
    double2 acc = make_double2(0, 0);
    for (int item = threadIdx.x; item < Vs * ncd; item += blockDim.x) {
        const int xs = item / ncd, i = item % ncd, h = i / nv, k = i % nv;
        const int X = xs + Vs * ct;
        const double2 *G = Gt + ((((size_t)X * at + tau) * 2 + h) * nv + k) * nv;
        const double2 *bb = b + ((size_t)r * M.Vc + X) * ncd + nv * h;
        double2 u = make_double2(0, 0);
        for (int l = 0; l < nv; ++l) u = zfma(u, G[l], bb[l]);
        const double2 av = a[((size_t)r * M.Vc + X) * ncd + i];
        const double sg = (gamma5 && h == 1) ? -1.0 : 1.0;
        acc.x += sg * (av.x * u.x + av.y * u.y);
        acc.y += sg * (av.x * u.y - av.y * u.x);
    }
    acc = block_reduce_z(acc, sh);
    if (threadIdx.x == 0) {
        part[((size_t)r * T + t) * 2] = acc.x;
        part[((size_t)r * T + t) * 2 + 1] = acc.y;
    }
}

// the same in double-float arithmetic: Gt as Ghi + Glo, b split once into the
// double-float layout, a split on the fly.  One CTA per (tile of CR RHS, t):
// each G row is read once for the CR RHS of the tile (the timeslice's G is
// 4 MB, read from L2 by every CTA of that timeslice).
template <int CR>
__global__ void __launch_bounds__(256, CR <= 4 ? 3 : 2) k_contract_coarse_t_dd(const float2 *Gh, const float2 *Gl, const double2 *a,
                                                              const float4 *b, int gamma5, double *part, MgGeom M,
                                                              int nrhs) {
    __shared__ double2 sh[32];
    const int r0 = blockIdx.x * CR, t = blockIdx.y, T = M.g.T;
    const int nr = nrhs - r0 < CR ? nrhs - r0 : CR;
    const int at = M.agg[3], nv = M.nv, ncd = M.ncd;
    const int Vs = M.cd[0] * M.cd[1] * M.cd[2];
    const int ct = t / at, tau = t % at;
    dd sre[CR], sim[CR];
#pragma unroll
    for (int q = 0; q < CR; ++q) { sre[q] = dd_make(0.f, 0.f); sim[q] = dd_make(0.f, 0.f); }
    for (int item = threadIdx.x; item < Vs * ncd; item += blockDim.x) {
        const int xs = item / ncd, i = item % ncd, h = i / nv, k = i % nv;
        const int X = xs + Vs * ct;
        const size_t g0 = ((((size_t)X * at + tau) * 2 + h) * nv + k) * nv;
        dd ure[CR], uim[CR];
#pragma unroll
        for (int q = 0; q < CR; ++q) { ure[q] = dd_make(0.f, 0.f); uim[q] = dd_make(0.f, 0.f); }
        for (int l = 0; l < nv; ++l) {
            const float2 mh = __ldg(Gh + g0 + l), ml = __ldg(Gl + g0 + l);
            const dd mr = dd_make(mh.x, ml.x), mi = dd_make(mh.y, ml.y);
#pragma unroll
            for (int q = 0; q < CR; ++q)
                if (q < nr) {
                    const float4 v = __ldg(b + ((size_t)(r0 + q) * M.Vc + X) * ncd + nv * h + l);
                    const dd vr = dd_make(v.x, v.z), vi = dd_make(v.y, v.w);
                    dd_fma(ure[q], mr, vr);
                    dd_fma(ure[q], -mi, vi);
                    dd_fma(uim[q], mr, vi);
                    dd_fma(uim[q], mi, vr);
                }
        }
#pragma unroll
        for (int q = 0; q < CR; ++q)
            if (q < nr) {
                const double2 av = a[((size_t)(r0 + q) * M.Vc + X) * ncd + i];
                dd ar = d2dd(av.x), ai = d2dd(av.y);
                if (gamma5 && h == 1) { ar = -ar; ai = -ai; }
                dd_fma(sre[q], ar, ure[q]);      // conj(a) u
                dd_fma(sre[q], ai, uim[q]);
                dd_fma(sim[q], ar, uim[q]);
                dd_fma(sim[q], -ai, ure[q]);
            }
    }
#pragma unroll
    for (int q = 0; q < CR; ++q) {
        double2 acc = make_double2(dd2d(sre[q]), dd2d(sim[q]));
        acc = block_reduce_z(acc, sh);
        if (threadIdx.x == 0 && q < nr) {
            part[((size_t)(r0 + q) * T + t) * 2] = acc.x;
            part[((size_t)(r0 + q) * T + t) * 2 + 1] = acc.y;
        }
    }
}

// Per-timeslice restriction: Rt[r][X][tau][i] = sum over the sites x of
// aggregate X at timeslice t0(X) + tau and the 6 components of half h(i) of
// conj(P_i(x)) v(x); the sum over tau is P^dag v.  DD: P as Phi + Plo and v
// in the double-float layout (ve, vo float4), else FP64 (P, ve, vo double).
// A thread takes one (X, tau, i) for RT right-hand sides, so that each P
// entry is read once per RT RHS (P is larger than L2).
template <bool DD, int RT>
__global__ void k_restrict_t(const double2 *P, const float2 *Ph, const float2 *Pl, const void *ve, const void *vo,
                             double2 *Rt, MgGeom M, int nrhs) {
    const int at = M.agg[3];
    const int ngrp = (nrhs + RT - 1) / RT;
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)ngrp * M.Vc * at * M.ncd) return;
    const int i = (int)(t % M.ncd);
    long rest = t / M.ncd;
    const int tau = (int)(rest % at);
    rest /= at;
    const int X = (int)(rest % M.Vc), r0 = (int)(rest / M.Vc) * RT;
    const int nr = nrhs - r0 < RT ? nrhs - r0 : RT;
    const int h = i / M.nv, k = i % M.nv;
    const int ns3 = M.agg[0] * M.agg[1] * M.agg[2];
    // origin of aggregate X at its timeslice tau; the sites of the aggregate
    // timeslice are walked with an incremental (dx, dy, dz) counter, x fastest
    int o[4];
    {
        int r = X;
        for (int m = 0; m < 4; ++m) { o[m] = (r % M.cd[m]) * M.agg[m]; r /= M.cd[m]; }
        o[3] += tau;
    }
    if constexpr (DD) {
        // software-pipelined over the (site, component) pairs: the P entry and
        // the RT field values of pair it + 1 are loaded before the arithmetic
        // of pair it, so every thread keeps one pair of loads in flight
        const size_t rstride = (size_t)12 * M.g.Vh;
        dd are[RT], aim[RT];
#pragma unroll
        for (int q = 0; q < RT; ++q) { are[q] = dd_make(0.f, 0.f); aim[q] = dd_make(0.f, 0.f); }
        int dx = 0, dy = 0, dz = 0, qc = 0;
        float2 mh, ml;
        float4 v[RT];
        auto load_pair = [&](int ddx, int ddy, int ddz, int qq, float2 &ph, float2 &pl, float4 (&w)[RT]) {
            const int c0 = o[0] + ddx, c1 = o[1] + ddy, c2 = o[2] + ddz;
            const int site = c0 + M.g.X * (c1 + M.g.Y * (c2 + M.g.Z * o[3]));
            const int par = (c0 + c1 + c2 + o[3]) & 1, sh = site >> 1;
            const int comp = 6 * h + qq;
            const size_t pi = (((size_t)par * M.g.Vh + sh) * 12 + comp) * M.nv + k;
            ph = __ldg(Ph + pi);
            pl = __ldg(Pl + pi);
            const float4 *base = (const float4 *)(par ? vo : ve) + ((size_t)r0 * 12 + comp) * M.g.Vh + sh;
#pragma unroll
            for (int q = 0; q < RT; ++q) w[q] = q < nr ? __ldg(base + q * rstride) : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        load_pair(0, 0, 0, 0, mh, ml, v);
        const int nit = ns3 * 6;
        for (int it = 0; it < nit; ++it) {
            float2 nmh = mh, nml = ml;
            float4 nv[RT];
#pragma unroll
            for (int q = 0; q < RT; ++q) nv[q] = v[q];
            if (it + 1 < nit) {
                if (++qc == 6) {
                    qc = 0;
                    if (++dx == M.agg[0]) { dx = 0; if (++dy == M.agg[1]) { dy = 0; ++dz; } }
                }
                load_pair(dx, dy, dz, qc, nmh, nml, nv);
            }
            const dd mr = dd_make(mh.x, ml.x), mi = dd_make(mh.y, ml.y);
#pragma unroll
            for (int q = 0; q < RT; ++q) {
                if (q < nr) {
                    const dd vr = dd_make(v[q].x, v[q].z), vi = dd_make(v[q].y, v[q].w);
                    dd_fma(are[q], mr, vr);  // conj(P) v
                    dd_fma(are[q], mi, vi);
                    dd_fma(aim[q], mr, vi);
                    dd_fma(aim[q], -mi, vr);
                }
            }
            mh = nmh; ml = nml;
#pragma unroll
            for (int q = 0; q < RT; ++q) v[q] = nv[q];
        }
#pragma unroll
        for (int q = 0; q < RT; ++q)
            if (q < nr)
                Rt[((((size_t)(r0 + q) * M.Vc + X) * at) + tau) * M.ncd + i] = make_double2(dd2d(are[q]), dd2d(aim[q]));
    } else {
        double2 acc[RT];
#pragma unroll
        for (int q = 0; q < RT; ++q) acc[q] = make_double2(0, 0);
        for (int j3 = 0; j3 < ns3; ++j3) {
            const int c0 = o[0] + j3 % M.agg[0], c1 = o[1] + (j3 / M.agg[0]) % M.agg[1];
            const int c2 = o[2] + j3 / (M.agg[0] * M.agg[1]);
            const int site = c0 + M.g.X * (c1 + M.g.Y * (c2 + M.g.Z * o[3]));
            const int par = (c0 + c1 + c2 + o[3]) & 1, sh = site >> 1;
            for (int qc = 0; qc < 6; ++qc) {
                const int comp = 6 * h + qc;
                const double2 pv = P[(((size_t)par * M.g.Vh + sh) * 12 + comp) * M.nv + k];
#pragma unroll
                for (int q = 0; q < RT; ++q)
                    if (q < nr) {
                        const size_t fi = ((size_t)(r0 + q) * 12 + comp) * M.g.Vh + sh;
                        acc[q] = zfma_conj(acc[q], pv, ((const double2 *)(par ? vo : ve))[fi]);
                    }
            }
        }
#pragma unroll
        for (int q = 0; q < RT; ++q)
            if (q < nr) Rt[((((size_t)(r0 + q) * M.Vc + X) * at) + tau) * M.ncd + i] = acc[q];
    }
}

// The same restriction for Rademacher noise (every entry +1 or -1, given as
// sign words: bit r of bits[(p Vh + s) 12 + comp] set where sample r0w + r is
// -1), with P as Phi + Plo: conj(P) eta is +/- conj(P), so each term is a
// double-float addition (TwoSum on the high parts, the low parts and the
// TwoSum errors summed in FP32 and folded into the pair once per site)
// instead of a double-float multiply-add, and the noise field is not read.
// A thread takes one (X, tau, i) for RT of the word's samples.
template <int RT>
__global__ void __launch_bounds__(128, RT <= 8 ? 6 : 4) k_restrict_t_sign(const float2 *Ph, const float2 *Pl,
                                                                          const unsigned long long *bits, double2 *Rt,
                                  MgGeom M, int nw, int r0w, int nrhs) {
    const int at = M.agg[3];
    const int ngrp = (nw + RT - 1) / RT;
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)ngrp * M.Vc * at * M.ncd) return;
    const int i = (int)(t % M.ncd);
    long rest = t / M.ncd;
    const int tau = (int)(rest % at);
    rest /= at;
    const int X = (int)(rest % M.Vc), rg = (int)(rest / M.Vc) * RT;
    const int nr = nw - rg < RT ? nw - rg : RT;
    const int h = i / M.nv, k = i % M.nv;
    int o[4];
    {
        int r = X;
        for (int m = 0; m < 4; ++m) { o[m] = (r % M.cd[m]) * M.agg[m]; r /= M.cd[m]; }
        o[3] += tau;
    }
    float reh[RT], rel[RT], imh[RT], iml[RT];
#pragma unroll
    for (int q = 0; q < RT; ++q) { reh[q] = 0.f; rel[q] = 0.f; imh[q] = 0.f; iml[q] = 0.f; }
    for (int dz = 0; dz < M.agg[2]; ++dz)
        for (int dy = 0; dy < M.agg[1]; ++dy)
            for (int dx = 0; dx < M.agg[0]; ++dx) {
                const int c0 = o[0] + dx, c1 = o[1] + dy, c2 = o[2] + dz;
                const int site = c0 + M.g.X * (c1 + M.g.Y * (c2 + M.g.Z * o[3]));
                const int par = (c0 + c1 + c2 + o[3]) & 1, sh = site >> 1;
                const size_t eo = ((size_t)par * M.g.Vh + sh) * 12 + 6 * h;
#pragma unroll 2
                for (int qc = 0; qc < 6; ++qc) {
                    const size_t pi = (eo + qc) * M.nv + k;
                    const float2 mh = __ldg(Ph + pi), ml = __ldg(Pl + pi);
                    const unsigned long long w = __ldg(bits + eo + qc) >> rg;
#pragma unroll
                    for (int q = 0; q < RT; ++q) {
                        // conj(P) eta: (Pr, -Pi) times +1 or -1
                        const float sr = ((w >> q) & 1) ? -1.f : 1.f;
                        float sv, e;
                        two_sum(reh[q], sr * mh.x, sv, e);
                        reh[q] = sv;
                        rel[q] = __fadd_rn(rel[q], __fadd_rn(e, sr * ml.x));
                        two_sum(imh[q], -sr * mh.y, sv, e);
                        imh[q] = sv;
                        iml[q] = __fadd_rn(iml[q], __fadd_rn(e, -sr * ml.y));
                    }
                }
#pragma unroll
                for (int q = 0; q < RT; ++q) {
                    float sv, e;
                    two_sum(reh[q], rel[q], sv, e); reh[q] = sv; rel[q] = e;
                    two_sum(imh[q], iml[q], sv, e); imh[q] = sv; iml[q] = e;
                }
            }
#pragma unroll
    for (int q = 0; q < RT; ++q)
        if (q < nr)
            Rt[((((size_t)(r0w + rg + q) * M.Vc + X) * at) + tau) * M.ncd + i] =
                make_double2(__dadd_rn((double)reh[q], (double)rel[q]), __dadd_rn((double)imh[q], (double)iml[q]));
}

// yc[r][X][i] = sum_tau Rt[r][X][tau][i], tau ascending
__global__ void k_sum_tau(const double2 *Rt, double2 *yc, MgGeom M, int nrhs) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)nrhs * M.Vc * M.ncd) return;
    const int i = (int)(t % M.ncd);
    const long rx = t / M.ncd;
    const int at = M.agg[3];
    double2 s = make_double2(0, 0);
    for (int tau = 0; tau < at; ++tau) {
        const double2 v = Rt[(rx * at + tau) * M.ncd + i];
        s.x += v.x;
        s.y += v.y;
    }
    yc[t] = s;
}

// part[r][t] = sum_{X in timeslice t / agg_t} sum_i s_h(i) conj(Rt[r][X][t % agg_t][i]) y[r][X][i]
__global__ void __launch_bounds__(256) k_contract_rt(const double2 *Rt, const double2 *y, int gamma5, double *part,
                                                     MgGeom M) {
    __shared__ double2 sh[32];
    const int r = blockIdx.x, t = blockIdx.y, T = M.g.T;
    const int at = M.agg[3], nv = M.nv, ncd = M.ncd;
    const int Vs = M.cd[0] * M.cd[1] * M.cd[2];
    const int ct = t / at, tau = t % at;
    double2 acc = make_double2(0, 0);
    for (int item = threadIdx.x; item < Vs * ncd; item += blockDim.x) {
        const int xs = item / ncd, i = item % ncd;
        const int X = xs + Vs * ct;
        const double2 rv = Rt[((((size_t)r * M.Vc + X) * at) + tau) * ncd + i];
        const double2 yv = y[((size_t)r * M.Vc + X) * ncd + i];
        const double sg = (gamma5 && i >= nv) ? -1.0 : 1.0;
        acc.x += sg * (rv.x * yv.x + rv.y * yv.y);
        acc.y += sg * (rv.x * yv.y - rv.y * yv.x);
    }
    acc = block_reduce_z(acc, sh);
    if (threadIdx.x == 0) {
        part[((size_t)r * T + t) * 2] = acc.x;
        part[((size_t)r * T + t) * 2 + 1] = acc.y;
    }
}

// coarse neighbour table: b = 0 self, 1+mu forward, 5+mu backward
__global__ void k_coarse_nbr(int *nbr, MgGeom M) {
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= M.Vc) return;
    int xc[4], r = X;
    for (int m = 0; m < 4; ++m) { xc[m] = r % M.cd[m]; r /= M.cd[m]; }
    nbr[X * 9] = X;
    for (int mu = 0; mu < 4; ++mu)
        for (int dir = 0; dir < 2; ++dir) {
            int y[4] = {xc[0], xc[1], xc[2], xc[3]};
            y[mu] = dir == 0 ? (y[mu] + 1) % M.cd[mu] : (y[mu] + M.cd[mu] - 1) % M.cd[mu];
            nbr[X * 9 + 1 + mu + 4 * dir] = y[0] + M.cd[0] * (y[1] + M.cd[1] * (y[2] + M.cd[2] * y[3]));
        }
}

// Block b of D_c at coarse site X (b = 0 .. 4: the site block and the forward
// ones; k_dc_backward derives the rest); one CTA per (X, b).  For each site x of
// the aggregate: A += P(x)^dag sum_hop coef [Gamma (x) U] P(y) over the hops
// x -> y of the block (the identity and the internal hops for b = 0), with
// P(.) the 12 x ncd restriction of the columns to one site: one ncd x ncd
// product per site instead of one per hop.  Shared memory: A (ncd^2), P(x),
// W = [Gamma (x) U] P(y), T1 and the hop sum Ws (12 x ncd each).
__global__ void k_assemble(const double2 *P, const double2 *U, int4 bc, double kappa, double2 *Dc, MgGeom M) {
    extern __shared__ double2 smem[];
    const int ncd = M.ncd, nv = M.nv;
    double2 *A = smem, *Px = A + ncd * ncd, *W = Px + 12 * ncd, *T1 = W + 12 * ncd, *Ws = T1 + 12 * ncd;
    const int X = blockIdx.x / 5, b = blockIdx.x % 5;   // the site block and the 4 forward ones
    const int nsite = M.agg[0] * M.agg[1] * M.agg[2] * M.agg[3];
    const int L[4] = {M.g.X, M.g.Y, M.g.Z, M.g.T};
    const int bcv[4] = {bc.x, bc.y, bc.z, bc.w};
    for (int e = threadIdx.x; e < ncd * ncd; e += blockDim.x) A[e] = make_double2(0, 0);
    // hop list: for b = 0 the identity (mu = -1) and internal hops; else the face hops of one direction.
    // The hops of block b that start at site x are summed into Ws = sum_hop coef [Gamma (x) U] P(y)
    // first, then A += P(x)^dag Ws once per site.
    for (int j = 0; j < nsite; ++j) {
        int c[4];
        agg_site(M, X, j, c);
        const int xs = lex(M.g, c);
        __syncthreads();
        for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) Ws[e] = make_double2(0, 0);
        bool any = false;
        for (int hop = -1; hop < 8; ++hop) {
            // hop -1: identity; 0..3 forward mu; 4..7 backward mu
            int mu = hop & 3, fwd = hop < 4;
            int y[4] = {c[0], c[1], c[2], c[3]};
            double sgn = 1.0;
            int blk;
            if (hop < 0) { blk = 0; }
            else {
                const int inside_f = (c[mu] % M.agg[mu]) != M.agg[mu] - 1;
                const int inside_b = (c[mu] % M.agg[mu]) != 0;
                if (fwd) {
                    y[mu] = c[mu] + 1 == L[mu] ? 0 : c[mu] + 1;
                    if (c[mu] == L[mu] - 1) sgn = bcv[mu];
                    blk = inside_f ? 0 : 1 + mu;
                } else {
                    y[mu] = c[mu] == 0 ? L[mu] - 1 : c[mu] - 1;
                    if (c[mu] == 0) sgn = bcv[mu];
                    blk = inside_b ? 0 : 5 + mu;
                }
            }
            if (blk != b) continue;
            any = true;
            const int ys = lex(M.g, y);
            __syncthreads();
            // P(y) restricted to the site (12 x ncd, zero outside each column's half)
            for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) {
                const int comp = e / ncd, i = e % ncd, h = i / nv, k = i % nv;
                W[e] = (comp / 6) == h ? P[pidx(M, ys, comp, k)] : make_double2(0, 0);
            }
            __syncthreads();
            double coef;
            if (hop >= 0) {
                // T1[s][a][i] = sum_b' U'[a][b'] P(y)[s][b'][i], U' = U_mu(x) (fwd) or U_mu(y)^dag (bwd)
                const double2 *u = U + ((size_t)mu * M.g.V + (fwd ? xs : ys)) * 9;
                for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) {
                    const int comp = e / ncd, i = e % ncd, s = comp / 3, a = comp % 3;
                    double2 acc = make_double2(0, 0);
                    // W is zero on the spins outside the half of i, and so is T1 there
                    if ((s >> 1) != i / nv) { T1[e] = acc; continue; }
                    for (int bb = 0; bb < 3; ++bb) {
                        double2 ul = fwd ? u[3 * a + bb] : make_double2(u[3 * bb + a].x, -u[3 * bb + a].y);
                        acc = zfma(acc, ul, W[(3 * s + bb) * ncd + i]);
                    }
                    T1[e] = acc;
                }
                __syncthreads();
                // W[s][a][i] = sum_s' (1 -/+ g_mu)[s][s'] T1[s'][a][i]
                for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) {
                    const int comp = e / ncd, i = e % ncd, s = comp / 3, a = comp % 3;
                    double2 acc = T1[e];
                    for (int sp = 0; sp < 4; ++sp) {
                        double2 gv = c_gamma[mu][s][sp];
                        if (fwd) { gv.x = -gv.x; gv.y = -gv.y; }
                        acc = zfma(acc, gv, T1[(3 * sp + a) * ncd + i]);
                    }
                    W[e] = acc;
                }
                __syncthreads();
                coef = -kappa * sgn;
            } else {
                coef = 1.0;
            }
            for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) {
                Ws[e].x += coef * W[e].x;
                Ws[e].y += coef * W[e].y;
            }
        }
        if (!any) continue;
        // P(x) restricted to the site, then A[i][j] += sum_comp conj(Px[comp][i]) Ws[comp][j]
        for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) {
            const int comp = e / ncd, i = e % ncd, h = i / nv, k = i % nv;
            Px[e] = (comp / 6) == h ? P[pidx(M, xs, comp, k)] : make_double2(0, 0);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < ncd * ncd; e += blockDim.x) {
            const int i = e / ncd, jj = e % ncd, c0 = 6 * (i / nv);
            double2 acc = make_double2(0, 0);
            // Px[comp][i] vanishes outside the half of i: the 6 components of that half
            for (int comp = c0; comp < c0 + 6; ++comp) acc = zfma_conj(acc, Px[comp * ncd + i], Ws[comp * ncd + jj]);
            A[e].x += acc.x;
            A[e].y += acc.y;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ncd * ncd; e += blockDim.x) Dc[((size_t)X * 9 + b) * ncd * ncd + e] = A[e];
}

// The same assembly in double-float arithmetic (FP32 pairs, ~2^-44 per
// operation; the FP64 rate is a small fraction of the FP32 one): P read as its
// FP32 pair copy (Ph + Pl), links split once per hop, the spin factor
// (1 -/+ gamma_mu) applied exactly (its entries are 0, +-1, +-i: sign flips and
// swaps), products and sums as in the FP64 kernel, in the same order.
struct cdd { dd re, im; };
__device__ __forceinline__ cdd cdd_zero() { cdd z; z.re = dd_make(0.f, 0.f); z.im = dd_make(0.f, 0.f); return z; }
__device__ __forceinline__ dd f64_to_dd(double x) {
    const float h = (float)x;
    return dd_make(h, (float)(x - (double)h));
}
// acc += a b (conj_a: conj(a) b)
template <bool CONJ_A>
__device__ __forceinline__ void cdd_fma(cdd &acc, const cdd &a, const cdd &b) {
    if (CONJ_A) {
        dd_fma(acc.re, a.re, b.re); dd_fma(acc.re, a.im, b.im);
        dd_fma(acc.im, a.re, b.im); dd_fma(acc.im, -a.im, b.re);
    } else {
        dd_fma(acc.re, a.re, b.re); dd_fma(acc.re, -a.im, b.im);
        dd_fma(acc.im, a.re, b.im); dd_fma(acc.im, a.im, b.re);
    }
}

__global__ void k_assemble_dd(const float2 *Ph, const float2 *Pl, const double2 *U, int4 bc, double kappa, double2 *Dc,
                              MgGeom M) {
    extern __shared__ cdd csm[];
    const int ncd = M.ncd, nv = M.nv;
    cdd *A = csm, *Px = A + ncd * ncd, *W = Px + 12 * ncd, *T1 = W + 12 * ncd, *Ws = T1 + 12 * ncd;
    const int X = blockIdx.x / 5, b = blockIdx.x % 5;   // the site block and the 4 forward ones
    const int nsite = M.agg[0] * M.agg[1] * M.agg[2] * M.agg[3];
    const int L[4] = {M.g.X, M.g.Y, M.g.Z, M.g.T};
    const int bcv[4] = {bc.x, bc.y, bc.z, bc.w};
    auto pload = [&](int site, int comp, int k) {
        const size_t q = pidx(M, site, comp, k);
        const float2 h = __ldg(Ph + q), l = __ldg(Pl + q);
        cdd r;
        r.re = dd_make(h.x, l.x);
        r.im = dd_make(h.y, l.y);
        return r;
    };
    for (int e = threadIdx.x; e < ncd * ncd; e += blockDim.x) A[e] = cdd_zero();
    for (int j = 0; j < nsite; ++j) {
        int c[4];
        agg_site(M, X, j, c);
        const int xs = lex(M.g, c);
        __syncthreads();
        for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) Ws[e] = cdd_zero();
        bool any = false;
        for (int hop = -1; hop < 8; ++hop) {
            int mu = hop & 3, fwd = hop < 4;
            int y[4] = {c[0], c[1], c[2], c[3]};
            double sgn = 1.0;
            int blk;
            if (hop < 0) { blk = 0; }
            else {
                const int inside_f = (c[mu] % M.agg[mu]) != M.agg[mu] - 1;
                const int inside_b = (c[mu] % M.agg[mu]) != 0;
                if (fwd) {
                    y[mu] = c[mu] + 1 == L[mu] ? 0 : c[mu] + 1;
                    if (c[mu] == L[mu] - 1) sgn = bcv[mu];
                    blk = inside_f ? 0 : 1 + mu;
                } else {
                    y[mu] = c[mu] == 0 ? L[mu] - 1 : c[mu] - 1;
                    if (c[mu] == 0) sgn = bcv[mu];
                    blk = inside_b ? 0 : 5 + mu;
                }
            }
            if (blk != b) continue;
            any = true;
            const int ys = lex(M.g, y);
            __syncthreads();
            for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) {
                const int comp = e / ncd, i = e % ncd, h = i / nv, k = i % nv;
                W[e] = (comp / 6) == h ? pload(ys, comp, k) : cdd_zero();
            }
            __syncthreads();
            if (hop >= 0) {
                const double2 *u = U + ((size_t)mu * M.g.V + (fwd ? xs : ys)) * 9;
                for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) {
                    const int comp = e / ncd, i = e % ncd, s = comp / 3, a = comp % 3;
                    cdd acc = cdd_zero();
                    if ((s >> 1) == i / nv) {   // W vanishes on the spins outside the half of i
                        for (int bb = 0; bb < 3; ++bb) {
                            const double2 uv = fwd ? u[3 * a + bb] : u[3 * bb + a];
                            cdd ul;
                            ul.re = f64_to_dd(uv.x);
                            ul.im = f64_to_dd(fwd ? uv.y : -uv.y);
                            cdd_fma<false>(acc, ul, W[(3 * s + bb) * ncd + i]);
                        }
                    }
                    T1[e] = acc;
                }
                __syncthreads();
                // W = (1 -/+ gamma_mu) T1: gamma entries are 0, +-1, +-i
                for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) {
                    const int comp = e / ncd, i = e % ncd, s = comp / 3, a = comp % 3;
                    cdd acc = T1[e];
                    for (int sp = 0; sp < 4; ++sp) {
                        double2 gv = c_gamma[mu][s][sp];
                        if (fwd) { gv.x = -gv.x; gv.y = -gv.y; }
                        const cdd t = T1[(3 * sp + a) * ncd + i];
                        if (gv.x > 0.5) { acc.re = acc.re + t.re; acc.im = acc.im + t.im; }
                        else if (gv.x < -0.5) { acc.re = acc.re - t.re; acc.im = acc.im - t.im; }
                        if (gv.y > 0.5) { acc.re = acc.re - t.im; acc.im = acc.im + t.re; }
                        else if (gv.y < -0.5) { acc.re = acc.re + t.im; acc.im = acc.im - t.re; }
                    }
                    W[e] = acc;
                }
                __syncthreads();
                const dd coef = f64_to_dd(-kappa * sgn);
                for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) {
                    dd_fma(Ws[e].re, coef, W[e].re);
                    dd_fma(Ws[e].im, coef, W[e].im);
                }
            } else {
                for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) {
                    Ws[e].re = Ws[e].re + W[e].re;
                    Ws[e].im = Ws[e].im + W[e].im;
                }
            }
        }
        if (!any) continue;
        for (int e = threadIdx.x; e < 12 * ncd; e += blockDim.x) {
            const int comp = e / ncd, i = e % ncd, h = i / nv, k = i % nv;
            Px[e] = (comp / 6) == h ? pload(xs, comp, k) : cdd_zero();
        }
        __syncthreads();
        for (int e = threadIdx.x; e < ncd * ncd; e += blockDim.x) {
            const int i = e / ncd, jj = e % ncd, c0 = 6 * (i / nv);
            cdd acc = cdd_zero();
            for (int comp = c0; comp < c0 + 6; ++comp) cdd_fma<true>(acc, Px[comp * ncd + i], Ws[comp * ncd + jj]);
            A[e].re = A[e].re + acc.re;
            A[e].im = A[e].im + acc.im;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ncd * ncd; e += blockDim.x)
        Dc[((size_t)X * 9 + b) * ncd * ncd + e] = make_double2(dd2d(A[e].re), dd2d(A[e].im));
}

// Chunked double-float assembly: the same blocks as k_assemble_dd with the
// sites of an aggregate that touch block b taken CH at a time.
//  * hop stage (all CH sites at once): W = P(y) restricted to the halves of
//    its columns, then Ws += coef [(1 -/+ gamma_mu) (U' (x) 1)] W, where for a
//    column of half h only one spin term survives (gamma_mu maps each half to
//    the other with one nonzero per row): 3 complex products per element;
//  * update stage: each thread keeps a 3 x 3 tile of the 48 x 48 block in
//    registers and adds sum_sites sum_{comp in its half} conj(Px) Ws.
// Two CTA barriers per hop instead of three per site and hop; no shared
// memory for the block itself.
template <int CH>
__global__ void __launch_bounds__(256) k_assemble_dd2(const float2 *Ph, const float2 *Pl, const double2 *U, int4 bc,
                                                      double kappa, double2 *Dc, MgGeom M) {
    extern __shared__ cdd csm[];
    const int ncd = M.ncd, nv = M.nv, NE = 12 * ncd;
    cdd *W = csm, *Ws = W + CH * NE, *Px = Ws + CH * NE;
    __shared__ int s_list[512];                 // aggregate sites (0..nsite-1) with a hop into block b
    __shared__ int s_n;
    __shared__ int s_ys[CH][9], s_xs[CH];       // per chunk site: neighbour of each hop (-1: none), the site
    __shared__ double s_coef[CH][9];
    __shared__ cdd s_u[CH][8][9];               // U' of each hop (U(x), or U(y)^dag backward), double-float
    __shared__ dd s_cd[CH][9];                  // the hop coefficients, double-float
    __shared__ int s_gp[4][4];                  // gamma partner spin and value (+-1, +-i) per (mu, s)
    __shared__ double2 s_gv[4][4];
    const int X = blockIdx.x / 5, b = blockIdx.x % 5;   // the site block and the 4 forward ones
    const int nsite = M.agg[0] * M.agg[1] * M.agg[2] * M.agg[3];
    const int L[4] = {M.g.X, M.g.Y, M.g.Z, M.g.T};
    const int bcv[4] = {bc.x, bc.y, bc.z, bc.w};
    if (threadIdx.x < 16) {
        const int mu = threadIdx.x >> 2, sp0 = threadIdx.x & 3;
        for (int sp = 0; sp < 4; ++sp) {
            const double2 g = c_gamma[mu][sp0][sp];
            if (g.x != 0.0 || g.y != 0.0) { s_gp[mu][sp0] = sp; s_gv[mu][sp0] = g; }
        }
    }
    if (threadIdx.x == 0) {
        int n = 0;
        for (int j = 0; j < nsite; ++j) {
            bool use = b == 0;
            if (!use) {
                int c[4];
                agg_site(M, X, j, c);
                const int mu = (b - 1) & 3;
                use = b <= 4 ? (c[mu] % M.agg[mu]) == M.agg[mu] - 1 : (c[mu] % M.agg[mu]) == 0;
            }
            if (use) s_list[n++] = j;
        }
        s_n = n;
    }
    __syncthreads();
    // the thread's 3 x 3 tile of the block, rows i0.., columns j0..
    const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
    const int i0 = 3 * ti, j0 = 3 * tj;
    const bool tile_on = i0 < ncd && j0 < ncd;
    cdd acc[3][3];
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
        for (int v = 0; v < 3; ++v) acc[u][v] = cdd_zero();
    auto pload = [&](int site, int comp, int k) {
        const size_t q = pidx(M, site, comp, k);
        const float2 hh = __ldg(Ph + q), ll = __ldg(Pl + q);
        cdd r;
        r.re = dd_make(hh.x, ll.x);
        r.im = dd_make(hh.y, ll.y);
        return r;
    };
    for (int base = 0; base < s_n; base += CH) {
        const int nc = min(CH, s_n - base);
        // hop table of the chunk
        if (threadIdx.x < CH * 9) {
            const int sl = threadIdx.x / 9, hop = threadIdx.x % 9 - 1;
            int ys = -1;
            double coef = 0.0;
            if (sl < nc) {
                int c[4];
                agg_site(M, X, s_list[base + sl], c);
                if (hop == -1) s_xs[sl] = lex(M.g, c);
                int mu = hop & 3, fwd = hop < 4;
                int y[4] = {c[0], c[1], c[2], c[3]};
                double sgn = 1.0;
                int blk;
                if (hop < 0) blk = 0;
                else {
                    const int inside_f = (c[mu] % M.agg[mu]) != M.agg[mu] - 1;
                    const int inside_b = (c[mu] % M.agg[mu]) != 0;
                    if (fwd) {
                        y[mu] = c[mu] + 1 == L[mu] ? 0 : c[mu] + 1;
                        if (c[mu] == L[mu] - 1) sgn = bcv[mu];
                        blk = inside_f ? 0 : 1 + mu;
                    } else {
                        y[mu] = c[mu] == 0 ? L[mu] - 1 : c[mu] - 1;
                        if (c[mu] == 0) sgn = bcv[mu];
                        blk = inside_b ? 0 : 5 + mu;
                    }
                }
                if (blk == b) { ys = lex(M.g, y); coef = hop < 0 ? 1.0 : -kappa * sgn; }
            }
            s_ys[sl][hop + 1] = ys;
            s_coef[sl][hop + 1] = coef;
        }
        for (int e = threadIdx.x; e < CH * NE; e += blockDim.x) Ws[e] = cdd_zero();
        __syncthreads();
        // the links and coefficients of the chunk's hops, split into FP32 pairs once
        // (the FP64 rate is a small fraction of the FP32 one)
        for (int e = threadIdx.x; e < CH * 9 * 10; e += blockDim.x) {
            const int sl = e / 90, r = e % 90, hop = r / 10 - 1, q = r % 10;
            const int ys = s_ys[sl][hop + 1];
            if (ys < 0) continue;
            if (q == 9) { s_cd[sl][hop + 1] = f64_to_dd(s_coef[sl][hop + 1]); continue; }
            if (hop < 0) continue;
            const int mu = hop & 3, fwd = hop < 4, a = q / 3, bb = q % 3;
            const double2 *u = U + ((size_t)mu * M.g.V + (fwd ? s_xs[sl] : ys)) * 9;
            const double2 uv = fwd ? u[3 * a + bb] : u[3 * bb + a];
            cdd ul;
            ul.re = f64_to_dd(uv.x);
            ul.im = f64_to_dd(fwd ? uv.y : -uv.y);
            s_u[sl][hop][q] = ul;
        }
        __syncthreads();
        for (int hop = -1; hop < 8; ++hop) {
            // a hop no site of the chunk takes is skipped by every thread alike
            bool used = false;
            for (int sl = 0; sl < CH; ++sl) used |= s_ys[sl][hop + 1] >= 0;
            if (!used) continue;
            // stage 1: W = P(y) of every chunk site that has this hop
            for (int e = threadIdx.x; e < CH * NE; e += blockDim.x) {
                const int sl = e / NE, r = e - sl * NE, comp = r / ncd, i = r - comp * ncd, h = i / nv, k = i - h * nv;
                const int ys = sl < nc ? s_ys[sl][hop + 1] : -1;
                W[e] = ys >= 0 && (comp / 6) == h ? pload(ys, comp, k) : cdd_zero();
            }
            __syncthreads();
            // stage 2: Ws += coef (1 -/+ gamma_mu) U' W, one surviving spin term per element
            for (int e = threadIdx.x; e < CH * NE; e += blockDim.x) {
                const int sl = e / NE, r = e - sl * NE, comp = r / ncd, i = r - comp * ncd;
                const int ys = sl < nc ? s_ys[sl][hop + 1] : -1;
                if (ys < 0) continue;
                const dd coef = s_cd[sl][hop + 1];
                const cdd *w = W + sl * NE;
                cdd out;
                if (hop < 0) {
                    out = w[r];
                } else {
                    const int mu = hop & 3, fwd = hop < 4, sg = comp / 3, a = comp % 3, h = i / nv;
                    const int sp = (sg >> 1) == h ? sg : s_gp[mu][sg];
                    cdd t = cdd_zero();
#pragma unroll
                    for (int bb = 0; bb < 3; ++bb) cdd_fma<false>(t, s_u[sl][hop][3 * a + bb], w[(3 * sp + bb) * ncd + i]);
                    if (sp == sg) {
                        out = t;
                    } else {   // (-/+ g) t with g in {+-1, +-i}
                        double2 gv = s_gv[mu][sg];
                        if (fwd) { gv.x = -gv.x; gv.y = -gv.y; }
                        if (gv.x > 0.5) out = t;
                        else if (gv.x < -0.5) { out.re = -t.re; out.im = -t.im; }
                        else if (gv.y > 0.5) { out.re = -t.im; out.im = t.re; }
                        else { out.re = t.im; out.im = -t.re; }
                    }
                }
                dd_fma(Ws[e].re, coef, out.re);
                dd_fma(Ws[e].im, coef, out.im);
            }
            __syncthreads();
        }
        // P(x) of the chunk sites, restricted to the halves of its columns
        for (int e = threadIdx.x; e < CH * NE; e += blockDim.x) {
            const int sl = e / NE, r = e - sl * NE, comp = r / ncd, i = r - comp * ncd, h = i / nv, k = i - h * nv;
            Px[e] = sl < nc && (comp / 6) == h ? pload(s_xs[sl], comp, k) : cdd_zero();
        }
        __syncthreads();
        if (tile_on) {
            const int c0 = 6 * (i0 / nv);
            for (int sl = 0; sl < nc; ++sl)
                for (int comp = c0; comp < c0 + 6; ++comp) {
                    const cdd *pr = Px + sl * NE + comp * ncd, *wr = Ws + sl * NE + comp * ncd;
                    cdd pa[3], wb[3];
#pragma unroll
                    for (int u = 0; u < 3; ++u) { pa[u] = pr[i0 + u]; wb[u] = wr[j0 + u]; }
#pragma unroll
                    for (int u = 0; u < 3; ++u)
#pragma unroll
                        for (int v = 0; v < 3; ++v) cdd_fma<true>(acc[u][v], pa[u], wb[v]);
                }
        }
        __syncthreads();
    }
    if (tile_on)
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
            for (int v = 0; v < 3; ++v)
                Dc[((size_t)X * 9 + b) * ncd * ncd + (size_t)(i0 + u) * ncd + j0 + v] =
                    make_double2(dd2d(acc[u][v].re), dd2d(acc[u][v].im));
}

// The backward blocks of D_c from the forward ones.  D is gamma5-hermitian
// and P keeps the two chirality halves apart (P gamma5c = gamma5 P, gamma5c =
// +1 on the first N_v coarse dofs of a site and -1 on the rest), so D_c =
// P^dag D P satisfies D_c^dag = gamma5c D_c gamma5c.  Block 5 + mu of X
// couples X to Y = X - mu, and Y's forward block 1 + mu couples Y to X, face
// by face (also when the coarse extent is 1 or 2), so
//   A_{5+mu}(X)[i][j] = s_i s_j conj(A_{1+mu}(Y)[j][i]).
// The assembly computes blocks 0 .. 4 only.
__global__ void k_dc_backward(double2 *Dc, const int *nbr, int Vc, int ncd, int nv) {
    const long n = (long)Vc * 4 * ncd * ncd;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
        const int j = (int)(e % ncd);
        long r = e / ncd;
        const int i = (int)(r % ncd);
        r /= ncd;
        const int mu = (int)(r % 4), X = (int)(r / 4);
        const int Y = nbr[X * 9 + 5 + mu];
        const double2 a = Dc[(((size_t)Y * 9 + 1 + mu) * ncd + j) * ncd + i];
        const double sg = ((i < nv) == (j < nv)) ? 1.0 : -1.0;
        Dc[(((size_t)X * 9 + 5 + mu) * ncd + i) * ncd + j] = make_double2(sg * a.x, -sg * a.y);
    }
}

__global__ void k_dc_to32(const double2 *Dc, float2 *D32, float2 *Dlo, long n) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const float hr = (float)Dc[i].x, hi = (float)Dc[i].y;
        D32[i] = make_float2(hr, hi);
        Dlo[i] = make_float2((float)(Dc[i].x - (double)hr), (float)(Dc[i].y - (double)hi));
    }
}

// FP64 residual of the coarse solves in double-float arithmetic (the block
// as Dc32 + Dclo, x split once into the double-float layout): y = a w + beta
// A x with the block products and the sums over j and the 9 blocks kept as
// float pairs (exact FMA errors, TwoSum), the final a w + beta acc in FP64.
// Each complex product m v = (a + ib)(c + id) takes three real products
// (Gauss): K1 += (a + b) c, K2 += a (d - c), K3 += b (c + d), and the
// outputs are Re = K1 - K3, Im = K1 + K2, so 36 instead of 48 FP32
// operations per term (the kernel is bound by instruction issue).  d - c and
// c + d are formed once per staged RHS element, a + b once per thread and j.
// One CTA per (X, 32-RHS tile), threads (i, rq); each of the 9 blocks is
// staged in shared memory by coalesced loads, transposed (column j
// contiguous, so the threads of a warp read consecutive words), together
// with the 32 RHS of its neighbour.
__global__ void __maxnreg__(56) k_coarse_apply_dd(const float2 *Dh, const float2 *Dl, const int *nbr,
                                                  const float4 *x, double2 *y, const double2 *w, double a,
                                                  double beta, int ncd, int Vc, int nrhs) {
    // one CTA per (X, tile of 32 RHS), threads (i, rq), rq < 8; thread (i, rq) takes the RHS
    // rq, rq + 8, rq + 16, rq + 24 of the tile, so each staged block element read from shared
    // memory (and its a + b) serves four RHS
    constexpr int NQ = 4, TILE = 8 * NQ;
    extern __shared__ float4 sm[];
    const int ld = ncd + 1;                                     // padded column stride
    float2 *Ah = (float2 *)sm, *Al = Ah + ncd * ld;
    float4 *xs4 = (float4 *)(Al + ncd * ld);                    // [TILE][ncd] (c.h, c.l, (d-c).h, (d-c).l)
    float2 *xs2 = (float2 *)(xs4 + TILE * ncd);                 // [TILE][ncd] ((c+d).h, (c+d).l)
    const int X = blockIdx.x, r0 = blockIdx.y * TILE;
    const int i = threadIdx.x % ncd, rq = threadIdx.x / ncd;
    const int nn = ncd * ncd;
    dd k1[NQ], k2[NQ], k3[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) { k1[q] = dd_make(0.f, 0.f); k2[q] = k1[q]; k3[q] = k1[q]; }
    for (int b = 0; b < 9; ++b) {
        const int nb = nbr[X * 9 + b];
        const size_t base = ((size_t)X * 9 + b) * nn;
        __syncthreads();
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int ei = e / ncd, ej = e - ei * ncd;          // row-major in global memory
            Ah[ej * ld + ei] = __ldg(Dh + base + e);
            Al[ej * ld + ei] = __ldg(Dl + base + e);
        }
        for (int e = threadIdx.x; e < TILE * ncd; e += blockDim.x) {
            const int er = e / ncd, ej = e - er * ncd;
            const float4 v = r0 + er < nrhs ? __ldg(x + ((size_t)(r0 + er) * Vc + nb) * ncd + ej)
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
            const dd c = dd_make(v.x, v.z), d = dd_make(v.y, v.w);
            const dd dmc = d - c, cpd = c + d;
            xs4[e] = make_float4(c.h, c.l, dmc.h, dmc.l);
            xs2[e] = make_float2(cpd.h, cpd.l);
        }
        __syncthreads();
        if (rq < 8) {
            for (int j = 0; j < ncd; ++j) {
                const float2 mh = Ah[j * ld + i], ml = Al[j * ld + i];
                const dd mr = dd_make(mh.x, ml.x), mi = dd_make(mh.y, ml.y), ms = mr + mi;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float4 v = xs4[(rq + 8 * q) * ncd + j];
                    const float2 u = xs2[(rq + 8 * q) * ncd + j];
                    dd_fma(k1[q], ms, dd_make(v.x, v.y));
                    dd_fma(k2[q], mr, dd_make(v.z, v.w));
                    dd_fma(k3[q], mi, dd_make(u.x, u.y));
                }
            }
        }
    }
    if (rq >= 8) return;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int r = r0 + rq + 8 * q;
        if (r >= nrhs) continue;
        const size_t o = ((size_t)r * Vc + X) * ncd + i;
        const double s1 = dd2d(k1[q]);
        double ore = beta * (s1 - dd2d(k3[q])), oim = beta * (s1 + dd2d(k2[q]));
        if (w) { ore += a * w[o].x; oim += a * w[o].y; }
        y[o] = make_double2(ore, oim);
    }
}

// FP32 coarse stencil y = A x for many RHS, tiled like k_coarse_apply_dd: one
// CTA per (X, 32-RHS tile), threads (i, rq), rq < 8, thread (i, rq) taking
// the RHS rq, rq + 8, rq + 16, rq + 24; each of the 9 blocks staged
// transposed in shared memory with the neighbour's 32 RHS.  The products and
// sums per output run in the order of k_coarse_apply<float2, float> (blocks
// b = 0..8, columns j = 0..ncd-1, the same four FMAs), so the two give the
// same bits.
__global__ void k_coarse_apply32t(const float2 *Dh, const int *nbr, const float2 *x, float2 *y, int ncd, int Vc,
                                  int nrhs) {
    constexpr int NQ = 4, TILE = 8 * NQ;
    extern __shared__ float2 sm2[];
    const int ld = ncd + 1;
    float2 *As = sm2, *xs = sm2 + ncd * ld;                     // [ncd][ld], [TILE][ncd]
    const int X = blockIdx.x, r0 = blockIdx.y * TILE;
    const int i = threadIdx.x % ncd, rq = threadIdx.x / ncd;
    const int nn = ncd * ncd;
    float are[NQ], aim[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) { are[q] = 0.f; aim[q] = 0.f; }
    for (int b = 0; b < 9; ++b) {
        const int nb = nbr[X * 9 + b];
        const size_t base = ((size_t)X * 9 + b) * nn;
        __syncthreads();
        for (int e = threadIdx.x; e < nn; e += blockDim.x) {
            const int ei = e / ncd, ej = e - ei * ncd;
            As[ej * ld + ei] = __ldg(Dh + base + e);
        }
        for (int e = threadIdx.x; e < TILE * ncd; e += blockDim.x) {
            const int er = e / ncd, ej = e - er * ncd;
            xs[e] = r0 + er < nrhs ? __ldg(x + ((size_t)(r0 + er) * Vc + nb) * ncd + ej) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (rq < 8) {
            for (int j = 0; j < ncd; ++j) {
                const float2 m = As[j * ld + i];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const float2 v = xs[(rq + 8 * q) * ncd + j];
                    are[q] = fmaf(m.x, v.x, are[q]); are[q] = fmaf(-m.y, v.y, are[q]);
                    aim[q] = fmaf(m.x, v.y, aim[q]); aim[q] = fmaf(m.y, v.x, aim[q]);
                }
            }
        }
    }
    if (rq >= 8) return;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int r = r0 + rq + 8 * q;
        if (r < nrhs) y[((size_t)r * Vc + X) * ncd + i] = make_float2(are[q], aim[q]);
    }
}

// ---- coarse stencil on CUDA cores (FP64 reference path and FP32) -----------
// y[rhs][X][i] = a*w[rhs][X][i] + beta * sum_b sum_j A_b(X)[i][j] x[rhs][nbr_b(X)][j]
// One CTA per (X, tile of 8 RHS), threads (i, r).
template <typename T2, typename R>
__global__ void k_coarse_apply(const T2 *Dc, const int *nbr, const T2 *x, T2 *y, const T2 *w, double a, double beta,
                               int ncd, int Vc, int nrhs) {
    const int X = blockIdx.x, r0 = blockIdx.y * 8;
    const int i = threadIdx.x % ncd, rr = threadIdx.x / ncd;
    const int r = r0 + rr;
    if (rr >= 8 || r >= nrhs) return;
    R are = 0, aim = 0;
    for (int b = 0; b < 9; ++b) {
        const int nb = nbr[X * 9 + b];
        const T2 *row = Dc + ((size_t)X * 9 + b) * ncd * ncd + (size_t)i * ncd;
        const T2 *xv = x + ((size_t)r * Vc + nb) * ncd;
        for (int j = 0; j < ncd; ++j) {
            const T2 m = row[j], v = xv[j];
            are = fma((R)m.x, (R)v.x, are); are = fma(-(R)m.y, (R)v.y, are);
            aim = fma((R)m.x, (R)v.y, aim); aim = fma((R)m.y, (R)v.x, aim);
        }
    }
    const size_t o = ((size_t)r * Vc + X) * ncd + i;
    R ore = (R)beta * are, oim = (R)beta * aim;
    if (w) { ore += (R)a * (R)w[o].x; oim += (R)a * (R)w[o].y; }
    T2 out;
    out.x = ore; out.y = oim;
    y[o] = out;
}

// ---- restriction / prolongation on eo FP64 fine fields ----------------------
// yc[rhs][X][nv*h + k] = sum_{x in X, spin in h, colour} conj(P[x][comp][k]) v[x][comp]
__global__ void k_restrict(const double2 *P, const double *ve, const double *vo, double2 *yc, MgGeom M, int nrhs) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)nrhs * M.Vc * M.ncd) return;
    const int i = (int)(t % M.ncd);
    const long rest = t / M.ncd;
    const int X = (int)(rest % M.Vc), r = (int)(rest / M.Vc);
    const int h = i / M.nv, k = i % M.nv;
    const int nsite = M.agg[0] * M.agg[1] * M.agg[2] * M.agg[3];
    double2 acc = make_double2(0, 0);
    for (int j = 0; j < nsite; ++j) {
        int c[4];
        agg_site(M, X, j, c);
        const int site = lex(M.g, c), par = (c[0] + c[1] + c[2] + c[3]) & 1, s = site >> 1;
        const double2 *f = (const double2 *)(par ? vo : ve) + (size_t)r * 12 * M.g.Vh;
        for (int q = 0; q < 6; ++q) {
            const int comp = 6 * h + q;
            acc = zfma_conj(acc, P[(((size_t)par * M.g.Vh + s) * 12 + comp) * M.nv + k], f[(size_t)comp * M.g.Vh + s]);
        }
    }
    yc[t] = acc;
}

// the same in double-float arithmetic: P as Phi + Plo, the fine fields split
// once into the double-float layout (ved, vod)
__global__ void k_restrict_dd(const float2 *Ph, const float2 *Pl, const float4 *ved, const float4 *vod, double2 *yc,
                              MgGeom M, int nrhs) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)nrhs * M.Vc * M.ncd) return;
    const int i = (int)(t % M.ncd);
    const long rest = t / M.ncd;
    const int X = (int)(rest % M.Vc), r = (int)(rest / M.Vc);
    const int h = i / M.nv, k = i % M.nv;
    const int nsite = M.agg[0] * M.agg[1] * M.agg[2] * M.agg[3];
    dd are = dd_make(0.f, 0.f), aim = dd_make(0.f, 0.f);
    for (int j = 0; j < nsite; ++j) {
        int c[4];
        agg_site(M, X, j, c);
        const int site = lex(M.g, c), par = (c[0] + c[1] + c[2] + c[3]) & 1, s = site >> 1;
        const float4 *f = (par ? vod : ved) + (size_t)r * 12 * M.g.Vh;
        for (int q = 0; q < 6; ++q) {
            const int comp = 6 * h + q;
            const size_t pi = (((size_t)par * M.g.Vh + s) * 12 + comp) * M.nv + k;
            const float2 mh = __ldg(Ph + pi), ml = __ldg(Pl + pi);
            const float4 v = __ldg(f + (size_t)comp * M.g.Vh + s);
            const dd mr = dd_make(mh.x, ml.x), mi = dd_make(mh.y, ml.y);
            const dd vr = dd_make(v.x, v.z), vi = dd_make(v.y, v.w);
            dd_fma(are, mr, vr);                 // conj(P) v
            dd_fma(are, mi, vi);
            dd_fma(aim, mr, vi);
            dd_fma(aim, -mi, vr);
        }
    }
    yc[t] = make_double2(dd2d(are), dd2d(aim));
}

// v[x][comp] = sum_k P[x][comp][k] yc[X][nv*h(comp) + k]   (overwrites v)
__global__ void k_prolong(const double2 *P, const double2 *yc, double *ve, double *vo, MgGeom M, int nrhs) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)nrhs * M.g.V * 12) return;
    const int comp = (int)(t % 12);
    const long rest = t / 12;
    const int site = (int)(rest % M.g.V), r = (int)(rest / M.g.V);
    int c[4];
    c[0] = site % M.g.X;
    int q = site / M.g.X;
    c[1] = q % M.g.Y; q /= M.g.Y;
    c[2] = q % M.g.Z; c[3] = q / M.g.Z;
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1, s = site >> 1;
    const int X = coarse_of(M, c), h = comp / 6;
    const double2 *pr = P + (((size_t)par * M.g.Vh + s) * 12 + comp) * M.nv;
    const double2 *yv = yc + ((size_t)r * M.Vc + X) * M.ncd + h * M.nv;
    double2 acc = make_double2(0, 0);
    for (int k = 0; k < M.nv; ++k) acc = zfma(acc, pr[k], yv[k]);
    double2 *f = (double2 *)(par ? vo : ve) + (size_t)r * 12 * M.g.Vh;
    f[(size_t)comp * M.g.Vh + s] = acc;
}

// the same in double-float arithmetic: P as Phi + Plo, yc split once into the
// double-float layout; within 2^-44 or so of the FP64 result, and not bound
// by the GPU's FP64 rate
__global__ void k_prolong_dd(const float2 *Ph, const float2 *Pl, const float4 *yc, double *ve, double *vo, MgGeom M,
                             int nrhs) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= (long)nrhs * M.g.V * 12) return;
    const int comp = (int)(t % 12);
    const long rest = t / 12;
    const int site = (int)(rest % M.g.V), r = (int)(rest / M.g.V);
    int c[4];
    c[0] = site % M.g.X;
    int q = site / M.g.X;
    c[1] = q % M.g.Y; q /= M.g.Y;
    c[2] = q % M.g.Z; c[3] = q / M.g.Z;
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1, s = site >> 1;
    const int X = coarse_of(M, c), h = comp / 6;
    const size_t pr = (((size_t)par * M.g.Vh + s) * 12 + comp) * M.nv;
    const float4 *yv = yc + ((size_t)r * M.Vc + X) * M.ncd + h * M.nv;
    dd are = dd_make(0.f, 0.f), aim = dd_make(0.f, 0.f);
    for (int k = 0; k < M.nv; ++k) {
        const float2 mh = __ldg(Ph + pr + k), ml = __ldg(Pl + pr + k);
        const float4 v = __ldg(yv + k);
        const dd mr = dd_make(mh.x, ml.x), mi = dd_make(mh.y, ml.y);
        const dd vr = dd_make(v.x, v.z), vi = dd_make(v.y, v.w);
        dd_fma(are, mr, vr);
        dd_fma(are, -mi, vi);
        dd_fma(aim, mr, vi);
        dd_fma(aim, mi, vr);
    }
    double2 *f = (double2 *)(par ? vo : ve) + (size_t)r * 12 * M.g.Vh;
    f[(size_t)comp * M.g.Vh + s] = make_double2(dd2d(are), dd2d(aim));
}

static MgGeom mg_geom(wd_ctx *c) {
    MgGeom M;
    M.g = c->g;
    for (int m = 0; m < 4; ++m) { M.agg[m] = c->mg->agg[m]; M.cd[m] = c->mg->cd[m]; }
    M.nv = c->mg->nv;
    M.ncd = c->mg->ncd;
    M.Vc = c->mg->Vc;
    return M;
}

Space coarse_space(wd_ctx *c) {
    Space s;
    s.units = (long)c->mg->Vc * c->mg->ncd / 12;
    s.flat = true;
    return s;
}

int coarse_apply64(wd_ctx *c, const double *x, double *y, const double *w, double a, double beta, int nrhs) {
    wd_mg *g = c->mg;
    dim3 grid(g->Vc, (nrhs + 7) / 8);
    int slot;
    prof_begin(c, WD_K_COARSE, 8.0 * g->ncd * g->ncd * 9.0 * g->Vc * nrhs, &slot);
    k_coarse_apply<double2, double><<<grid, g->ncd * 8, 0, c->st>>>(g->Dc, g->nbr, (const double2 *)x, (double2 *)y,
                                                                   (const double2 *)w, a, beta, g->ncd, g->Vc, nrhs);
    prof_end(c, slot);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// y = a*w + beta * D_c x on FP64 vectors in double-float arithmetic
int coarse_apply_dd(wd_ctx *c, const double *x, double *y, const double *w, double a, double beta, int nrhs) {
    wd_mg *g = c->mg;
    const long n = (long)g->Vc * g->ncd * nrhs;
    void *xd;
    WD_TRY(ws_get(c, "coarse.xdd", (size_t)n * sizeof(float4), &xd));
    WD_CUDA(launch_to_ddl(x, xd, n, c->st));
    dim3 grid(g->Vc, (nrhs + 31) / 32);
    const size_t nld = (size_t)g->ncd * (g->ncd + 1);
    const size_t smem = 2 * nld * sizeof(float2) + (size_t)32 * g->ncd * (sizeof(float4) + sizeof(float2));
    WD_CUDA(cudaFuncSetAttribute(k_coarse_apply_dd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // three 74.5 KB CTAs per SM (2N_v = 48) fit only in the largest shared-memory carveout
    WD_CUDA(cudaFuncSetAttribute(k_coarse_apply_dd, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared));
    k_coarse_apply_dd<<<grid, g->ncd * 8, smem, c->st>>>(g->Dc32, g->Dclo, g->nbr, (const float4 *)xd, (double2 *)y,
                                                         (const double2 *)w, a, beta, g->ncd, g->Vc, nrhs);
    c->launches += 2;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// any 9-point block stencil (blocks [V][9][n][n], neighbour table [V][9]):
// y = a*w + beta * A x, FP64 (the third level uses it)
int block_stencil_apply64(wd_ctx *c, const double2 *A, const int *nbr, int n, int V, const double *x, double *y,
                          const double *w, double a, double beta, int nrhs) {
    dim3 grid(V, (nrhs + 7) / 8);
    k_coarse_apply<double2, double><<<grid, n * 8, 0, c->st>>>(A, nbr, (const double2 *)x, (double2 *)y,
                                                              (const double2 *)w, a, beta, n, V, nrhs);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int coarse_apply32(wd_ctx *c, const float *x, float *y, int nrhs) {
    wd_mg *g = c->mg;
    int slot;
    prof_begin(c, WD_K_COARSE, 8.0 * g->ncd * g->ncd * 9.0 * g->Vc * nrhs, &slot);
    if (nrhs >= 16) {
        dim3 grid(g->Vc, (nrhs + 31) / 32);
        const size_t smem = ((size_t)g->ncd * (g->ncd + 1) + 32 * (size_t)g->ncd) * sizeof(float2);
        WD_CUDA(cudaFuncSetAttribute(k_coarse_apply32t, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_coarse_apply32t<<<grid, g->ncd * 8, smem, c->st>>>(g->Dc32, g->nbr, (const float2 *)x, (float2 *)y, g->ncd,
                                                            g->Vc, nrhs);
    } else {
        dim3 grid(g->Vc, (nrhs + 7) / 8);
        k_coarse_apply<float2, float><<<grid, g->ncd * 8, 0, c->st>>>(g->Dc32, g->nbr, (const float2 *)x, (float2 *)y,
                                                                      nullptr, 0.0, 1.0, g->ncd, g->Vc, nrhs);
    }
    prof_end(c, slot);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int mg_restrict_eo(wd_ctx *c, const double *ve, const double *vo, double *yc, int nrhs, bool dd_ok) {
    MgGeom M = mg_geom(c);
    const long n = (long)nrhs * M.Vc * M.ncd;
    if (dd_ok && c->outer == PDD && c->mg->Phi) {
        void *ved, *vod;
        const long nf = 12L * M.g.Vh * nrhs;
        WD_TRY(ws_get(c, "mg.vedd", (size_t)nf * sizeof(float4), &ved));
        WD_TRY(ws_get(c, "mg.vodd", (size_t)nf * sizeof(float4), &vod));
        WD_CUDA(launch_to_ddl(ve, ved, nf, c->st));
        WD_CUDA(launch_to_ddl(vo, vod, nf, c->st));
        k_restrict_dd<<<(unsigned)((n + 127) / 128), 128, 0, c->st>>>(c->mg->Phi, c->mg->Plo, (const float4 *)ved,
                                                                      (const float4 *)vod, (double2 *)yc, M, nrhs);
        c->launches += 3;
    } else {
        k_restrict<<<(unsigned)((n + 127) / 128), 128, 0, c->st>>>(c->mg->P, ve, vo, (double2 *)yc, M, nrhs);
        c->launches++;
    }
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int mg_prolong_eo(wd_ctx *c, const double *yc, double *ve, double *vo, int nrhs, bool dd_ok) {
    MgGeom M = mg_geom(c);
    const long n = (long)nrhs * M.g.V * 12;
    if (dd_ok && c->outer == PDD && c->mg->Phi) {
        // double-float: the prolongated fields carry the FP64 values to ~2^-44
        void *yd;
        const long nc = (long)nrhs * M.Vc * M.ncd;
        WD_TRY(ws_get(c, "mg.ydd", (size_t)nc * sizeof(float4), &yd));
        WD_CUDA(launch_to_ddl(yc, yd, nc, c->st));
        k_prolong_dd<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>(c->mg->Phi, c->mg->Plo, (const float4 *)yd, ve,
                                                                     vo, M, nrhs);
        c->launches += 2;
    } else {
        k_prolong<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>(c->mg->P, (const double2 *)yc, ve, vo, M, nrhs);
        c->launches++;
    }
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// ---- coarse solves ------------------------------------------------------------
int mg_contract_coarse_t(wd_ctx *c, const double *a, const double *b, int gamma5, int nrhs, double *part) {
    wd_mg *g = c->mg;
    if (!g || !g->Gt) { set_error("coarse contraction: no multigrid setup"); return WD_EINVAL; }
    if (nrhs <= 0) return WD_OK;
    const MgGeom M = mg_geom(c);
    if (c->outer == PDD && g->Ghi) {
        // double-float arithmetic (the FP64 rate is a small fraction of the FP32 one)
        void *bd;
        const long nc = (long)nrhs * M.Vc * M.ncd;
        WD_TRY(ws_get(c, "mg.cdd", (size_t)nc * sizeof(float4), &bd));
        WD_CUDA(launch_to_ddl(b, bd, nc, c->st));
        // RHS per CTA tile: 4 (79 registers, three CTAs of 256 threads per SM)
        // beats 8 (125 registers, two CTAs): the kernel is bound by the latency
        // of its loads (ncu: issue 52 %, long-scoreboard stalls), not by the G
        // rows it reads once per tile.  Two-level step on 24^3x48: 0.366 ->
        // 0.361 s.  WD_CONTRACT_CR = 8 restores the larger tile.
        int cr = 4;
        if (const char *e = getenv("WD_CONTRACT_CR")) cr = atoi(e) == 8 ? 8 : 4;
        if (cr == 4)
            k_contract_coarse_t_dd<4><<<dim3((nrhs + 3) / 4, c->g.T), 256, 0, c->st>>>(
                g->Ghi, g->Glo, (const double2 *)a, (const float4 *)bd, gamma5, part, M, nrhs);
        else
            k_contract_coarse_t_dd<8><<<dim3((nrhs + 7) / 8, c->g.T), 256, 0, c->st>>>(
                g->Ghi, g->Glo, (const double2 *)a, (const float4 *)bd, gamma5, part, M, nrhs);
        c->launches += 2;
    } else {
        k_contract_coarse_t<<<dim3(nrhs, c->g.T), 256, 0, c->st>>>(g->Gt, (const double2 *)a, (const double2 *)b,
                                                                  gamma5, part, M);
        c->launches++;
    }
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int mg_restrict_t_eo(wd_ctx *c, const double *ve, const double *vo, double *Rt, double *yc, int nrhs) {
    const MgGeom M = mg_geom(c);
    // RHS per thread: each P entry is read once per RT RHS.  Measured on the
    // 24^3x48 two-level step (64 level-1 samples): 8 is fastest; 16 (and 32,
    // which spills) lose more to register pressure than they gain in P traffic
    int RT = 8;
    if (const char *e = getenv("WD_RESTRICT_RT")) {   // tuning override: 8 or 16
        const int r = atoi(e);
        if (r == 8 || r == 16) RT = r;
    }
    const long n = (long)((nrhs + RT - 1) / RT) * M.Vc * M.agg[3] * M.ncd;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    if (c->outer == PDD && c->mg->Phi) {
        void *ved, *vod;
        const long nf = 12L * M.g.Vh * nrhs;
        WD_TRY(ws_get(c, "mg.vedd", (size_t)nf * sizeof(float4), &ved));
        WD_TRY(ws_get(c, "mg.vodd", (size_t)nf * sizeof(float4), &vod));
        WD_CUDA(launch_to_ddl(ve, ved, nf, c->st));
        WD_CUDA(launch_to_ddl(vo, vod, nf, c->st));
#define WD_RT_CASE(R)                                                                                          \
        if (RT == R)                                                                                           \
            k_restrict_t<true, R><<<blocks, 128, 0, c->st>>>(nullptr, c->mg->Phi, c->mg->Plo, ved, vod, (double2 *)Rt, M, nrhs);
        WD_RT_CASE(8) WD_RT_CASE(16)
#undef WD_RT_CASE
        c->launches += 3;
    } else {
#define WD_RT_CASE(R)                                                                                          \
        if (RT == R)                                                                                           \
            k_restrict_t<false, R><<<blocks, 128, 0, c->st>>>(c->mg->P, nullptr, nullptr, ve, vo, (double2 *)Rt, M, nrhs);
        WD_RT_CASE(8) WD_RT_CASE(16)
#undef WD_RT_CASE
        c->launches++;
    }
    const long nc = (long)nrhs * M.Vc * M.ncd;
    k_sum_tau<<<(unsigned)((nc + 255) / 256), 256, 0, c->st>>>((const double2 *)Rt, (double2 *)yc, M, nrhs);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int gen_noise_signs(wd_ctx *c, uint64_t seed, int sample0, int nrhs, unsigned long long *bits);   // wd_estim.cu

int mg_restrict_t_noise(wd_ctx *c, uint64_t seed, int sample0, const double *ve, const double *vo, double *Rt,
                        double *yc, int nrhs) {
    if (!(c->outer == PDD && c->mg->Phi)) return mg_restrict_t_eo(c, ve, vo, Rt, yc, nrhs);
    const MgGeom M = mg_geom(c);
    // samples per thread: each P entry is read once per RT samples
    int RT = 16;
    if (const char *e = getenv("WD_RESTRICT_RT")) {   // tuning override: 8, 16 or 32
        const int r = atoi(e);
        if (r == 8 || r == 16 || r == 32) RT = r;
    }
    unsigned long long *bits;
    WD_TRY(ws_get(c, "mg.signs", sizeof(unsigned long long) * 12 * (size_t)M.g.V, (void **)&bits));
    for (int w0 = 0; w0 < nrhs; w0 += 64) {
        const int nw = nrhs - w0 < 64 ? nrhs - w0 : 64;
        WD_TRY(gen_noise_signs(c, seed, sample0 + w0, nw, bits));
        const long n = (long)((nw + RT - 1) / RT) * M.Vc * M.agg[3] * M.ncd;
        const unsigned blocks = (unsigned)((n + 127) / 128);
        if (RT == 32) k_restrict_t_sign<32><<<blocks, 128, 0, c->st>>>(c->mg->Phi, c->mg->Plo, bits, (double2 *)Rt, M, nw, w0, nrhs);
        else if (RT == 8) k_restrict_t_sign<8><<<blocks, 128, 0, c->st>>>(c->mg->Phi, c->mg->Plo, bits, (double2 *)Rt, M, nw, w0, nrhs);
        else k_restrict_t_sign<16><<<blocks, 128, 0, c->st>>>(c->mg->Phi, c->mg->Plo, bits, (double2 *)Rt, M, nw, w0, nrhs);
        c->launches++;
        WD_CUDA(cudaGetLastError());
    }
    const long nc = (long)nrhs * M.Vc * M.ncd;
    k_sum_tau<<<(unsigned)((nc + 255) / 256), 256, 0, c->st>>>((const double2 *)Rt, (double2 *)yc, M, nrhs);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

int mg_contract_rt(wd_ctx *c, const double *Rt, const double *y, int gamma5, int nrhs, double *part) {
    if (nrhs <= 0) return WD_OK;
    k_contract_rt<<<dim3(nrhs, c->g.T), 256, 0, c->st>>>((const double2 *)Rt, (const double2 *)y, gamma5, part,
                                                        mg_geom(c));
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// x an FP32 coarse field; split = false: x and the blocks rounded to BF16;
// true: both as BF16 pairs (hi + lo, ~16 significant bits)
int coarse_tc_apply(wd_ctx *c, const void *x, float *y, int nrhs, bool split = false);   // wd_coarse_tc.cu
int coarse_tc_check(wd_ctx *c);
int coarse_tc_build(wd_ctx *c);
bool coarse_tc_ok(wd_ctx *c);

static int cop64(wd_ctx *c, const void *in, void *out, int nrhs, void *) {
    return coarse_apply64(c, (const double *)in, (double *)out, nullptr, 0.0, 1.0, nrhs);
}
static int cop32(wd_ctx *c, const void *in, void *out, int nrhs, void *) {
    return coarse_apply32(c, (const float *)in, (float *)out, nrhs);
}
// inner operator of the mixed coarse solves on the tensor cores: FP32 Krylov
// vectors, the vectors and the blocks both multiplied as BF16 pairs (hi + lo,
// ~16 significant bits), so that an inner solve can go to 1e-5 and the outer
// loop needs two FP64 residuals instead of four or five
static int coptc_split(wd_ctx *c, const void *in, void *out, int nrhs, void *) {
    return coarse_tc_apply(c, in, (float *)out, nrhs, true);
}
// r = b - D_c x; u (nullable) points at a flag: nonzero = double-float arithmetic
static int cres64(wd_ctx *c, const double *b, const double *x, double *r, int nrhs, void *u) {
    if (u && *(const int *)u) return coarse_apply_dd(c, x, r, b, 1.0, -1.0, nrhs);
    return coarse_apply64(c, x, r, b, 1.0, -1.0, nrhs);
}

// x = D_c^{-1} b on coarse FP64 vectors [nrhs][Vc][ncd]
int coarse_solve(wd_ctx *c, const double *b, double *x, int nrhs, double tol, int prec, int max_iter,
                 double *resid_out) {
    const Space sp = coarse_space(c);
    double *bn2;
    WD_TRY(ws_get(c, "cs.bn2", sizeof(double) * nrhs, (void **)&bn2));
    WD_TRY(blas_norm2(c, sp, P64, b, nrhs, bn2));
    std::vector<double> bnorm2(nrhs);
    WD_CUDA(cudaMemcpyAsync(bnorm2.data(), bn2, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaStreamSynchronize(c->st));
    Problem P;
    P.sp = sp;
    P.op64 = cop64; P.u64 = nullptr;
    // mixed: BF16-pair operands on the tensor cores when available, else the
    // FP32 blocks on the CUDA cores
    const bool tc = prec != P64 && coarse_tc_ok(c) && c->mg->Wlo;
    P.oplo = tc ? coptc_split : cop32; P.ulo = nullptr;
    // once the residual is small, r <- r - D_c e with the FP32 blocks on the
    // CUDA cores instead of a double-float residual: the FP32 product is off by
    // a few 1e-8 of |D_c| |e| (rounded blocks, FP32 sums of 9 x ncd terms);
    // 1e-6 of |r| bounds it with the norm of D_c^{-1} folded in
    if (prec != P64) { P.opupd = cop32; P.upd_err = 1e-6; }
    // the FP64 residuals of the mixed solves in double-float arithmetic, as on
    // the fine lattice (~2^-44 normwise), unless the tolerance asks for more
    int use_dd = prec != P64 && tol >= 1e-12 && c->outer == PDD;
    P.res64 = cres64; P.ures = &use_dd;
    P.tag = "coarse";
    const int inner = P32;
    std::vector<int> iters;
    std::vector<double> last;
    int s = dc_solve(c, P, b, x, nrhs, bn2, bnorm2, tol, prec == P64 ? P64 : inner, max_iter, iters, last);
    if (tc) WD_TRY(coarse_tc_check(c));
    if (resid_out) {
        double *r, *n2;
        WD_TRY(ws_get(c, "cs.r", space_bytes(sp, P64, nrhs), (void **)&r));
        WD_TRY(ws_get(c, "cs.n2", sizeof(double) * nrhs, (void **)&n2));
        WD_TRY(cres64(c, b, x, r, nrhs, nullptr));
        WD_TRY(blas_norm2(c, sp, P64, r, nrhs, n2));
        std::vector<double> h(nrhs);
        WD_CUDA(cudaMemcpyAsync(h.data(), n2, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->st));
        WD_CUDA(cudaStreamSynchronize(c->st));
        for (int i = 0; i < nrhs; ++i) resid_out[i] = bnorm2[i] > 0 ? sqrt(h[i] / bnorm2[i]) : 0.0;
    }
    return s;
}

}  // namespace wd

using namespace wd;

void wd_mg3_free(wd_ctx *c);   // wd_mg3.cu

void wd_mg_free(wd_ctx *c) {
    wd_mg3_free(c);               // the third level is built on this one
    if (!c || !c->mg) return;
    wd_mg *g = c->mg;
    cudaFree(g->P);
    cudaFree(g->Dc);
    cudaFree(g->nbr);
    if (g->Wtc) cudaFree(g->Wtc);
    if (g->Wlo) cudaFree(g->Wlo);
    if (g->Dc32) cudaFree(g->Dc32);
    if (g->Dclo) cudaFree(g->Dclo);
    if (g->Phi) cudaFree(g->Phi);
    if (g->Plo) cudaFree(g->Plo);
    if (g->Gt) cudaFree(g->Gt);
    if (g->Ghi) cudaFree(g->Ghi);
    if (g->Glo) cudaFree(g->Glo);
    delete g;
    c->mg = nullptr;
}

namespace wd {
int mg_generate_tv(wd_ctx *c, int nv, int iters, uint64_t seed, double *tv_dev);   // wd_mlmc.cu
}

extern "C" int wd_mg_setup(wd_ctx *c, const double *tv, int nv, const int agg[4], int tv_iters, uint64_t seed) {
    if (!c || !agg || nv < 1 || nv % 6 != 0) {
        set_error("wd_mg_setup: bad argument (nv must be a positive multiple of 6)");
        return WD_EINVAL;
    }
    int nsite = 1;
    for (int m = 0; m < 4; ++m) {
        if (agg[m] < 1 || c->dims[m] % agg[m]) { set_error("wd_mg_setup: aggregate extent %d does not divide %d", agg[m], c->dims[m]); return WD_EINVAL; }
        nsite *= agg[m];
    }
    if (nv > 6 * nsite) { set_error("wd_mg_setup: nv > 6 * aggregate volume"); return WD_EINVAL; }
    const int ncd = 2 * nv;
    const size_t smem = sizeof(double2) * ((size_t)ncd * ncd + 4 * 12 * ncd);
    if (smem > 227 * 1024) { set_error("wd_mg_setup: nv too large for the block assembly"); return WD_ENOTSUP; }
    // A new setup with the geometry of the current one (the same N_v and
    // aggregates, e.g. the next gauge configuration) overwrites its buffers in
    // place: ~8 GB at 24^3x48 that need not be freed and mapped again.  The
    // third level, built on the old operator, goes.
    const bool reuse = c->mg && c->mg->nv == nv && c->mg->agg[0] == agg[0] && c->mg->agg[1] == agg[1] &&
                       c->mg->agg[2] == agg[2] && c->mg->agg[3] == agg[3];
    if (reuse) wd_mg3_free(c);
    else wd_mg_free(c);
    wd_mg *g = reuse ? c->mg : new wd_mg();
    if (!reuse) memset(g, 0, sizeof(*g));
    c->mg = g;
    g->nv = nv;
    g->ncd = ncd;
    g->Vc = 1;
    for (int m = 0; m < 4; ++m) { g->agg[m] = agg[m]; g->cd[m] = c->dims[m] / agg[m]; g->Vc *= g->cd[m]; }
    const size_t nP = (size_t)c->g.V * 12 * nv;
    const size_t nD = (size_t)g->Vc * 9 * ncd * ncd;
    if (!reuse && (cudaMalloc(&g->P, nP * sizeof(double2)) != cudaSuccess || cudaMalloc(&g->Dc, nD * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&g->nbr, sizeof(int) * 9 * g->Vc) != cudaSuccess || cudaMalloc(&g->Dc32, nD * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&g->Dclo, nD * sizeof(float2)) != cudaSuccess || cudaMalloc(&g->Phi, nP * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&g->Plo, nP * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&g->Gt, sizeof(double2) * (size_t)g->Vc * agg[3] * 2 * nv * nv) != cudaSuccess ||
        cudaMalloc(&g->Ghi, sizeof(float2) * (size_t)g->Vc * agg[3] * 2 * nv * nv) != cudaSuccess ||
        cudaMalloc(&g->Glo, sizeof(float2) * (size_t)g->Vc * agg[3] * 2 * nv * nv) != cudaSuccess)) {
        cudaGetLastError();
        wd_mg_free(c);
        set_error("wd_mg_setup: allocation failed");
        return WD_ENOMEM;
    }
    MgGeom M = mg_geom(c);
    // WD_VERBOSE: the wall time of each phase (the stream synchronised at the
    // phase ends, so only then)
    const bool verbose = getenv("WD_VERBOSE") != nullptr;
    auto t_last = std::chrono::steady_clock::now();
    auto phase = [&](const char *name) {
        if (!verbose) return;
        cudaStreamSynchronize(c->st);
        const auto now = std::chrono::steady_clock::now();
        fprintf(stderr, "[wd] setup %-24s %8.2f ms\n", name,
                std::chrono::duration<double, std::milli>(now - t_last).count());
        t_last = now;
    };
    phase("allocation");
    double *tvd;
    WD_TRY(ws_get(c, "mg.tv", nP * sizeof(double2), (void **)&tvd));
    if (tv) {
        WD_CUDA(cudaMemcpyAsync(tvd, tv, nP * sizeof(double2), cudaMemcpyHostToDevice, c->st));
    } else {
        WD_TRY(mg_generate_tv(c, nv, tv_iters, seed, tvd));
    }
    phase("test vectors");
    k_tv_to_P<<<(unsigned)((nP + 255) / 256), 256, 0, c->st>>>((const double2 *)tvd, g->P, M);
    // block MGS on a column-major copy of the blocks (coalesced passes), kept in
    // the test-vector workspace, which P has been built from (same size)
    k_mgs_gather<<<1184, 256, 0, c->st>>>(g->P, (double2 *)tvd, M, 1);
    // one warp per block where four columns fit in shared memory, else one CTA per block
    const size_t mgs_smem = (size_t)4 * nsite * 6 * sizeof(double2);
    if (mgs_smem <= 200 * 1024) {
        WD_CUDA(cudaFuncSetAttribute(k_block_mgs_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mgs_smem));
        k_block_mgs_warp<<<(2 * g->Vc + 3) / 4, 128, mgs_smem, c->st>>>((double2 *)tvd, M, 2 * g->Vc);
    } else {
        k_block_mgs_cm<<<2 * g->Vc, 256, 0, c->st>>>((double2 *)tvd, M);
    }
    k_mgs_gather<<<1184, 256, 0, c->st>>>(g->P, (double2 *)tvd, M, 0);
    phase("block MGS");
    k_coarse_nbr<<<(g->Vc + 127) / 128, 128, 0, c->st>>>(g->nbr, M);
    k_dc_to32<<<1184, 256, 0, c->st>>>(g->P, g->Phi, g->Plo, (long)nP);
    if (c->outer == PDD) k_gram_t_dd<<<g->Vc * agg[3] * 2, 256, 0, c->st>>>(g->Phi, g->Plo, g->Gt, M);
    else k_gram_t<<<g->Vc * agg[3] * 2, 256, 0, c->st>>>(g->P, g->Gt, M);
    phase("P pairs, Gram matrices");
    double2 hg[4][4][4];
    host_gamma(hg);
    WD_CUDA(cudaMemcpyToSymbolAsync(c_gamma, hg, sizeof(hg), 0, cudaMemcpyHostToDevice, c->st));
    // links in lexicographic FP64 (kept by gauge ingest)
    void *ulex = nullptr;
    {
        auto it = c->bufs.find("gauge.lex");
        if (it == c->bufs.end()) { set_error("wd_mg_setup: links not resident"); return WD_ECUDA; }
        ulex = it->second.first;
    }
    const int4 bc = make_int4(c->bc[0], c->bc[1], c->bc[2], c->bc[3]);
    if (c->outer == PDD) {
        // double-float Galerkin assembly (FP32 pairs; ~2^-44 per operation)
        if (ncd <= 48 && nsite <= 512) {
            // chunks of CH sites; the 48 x 48 block in 3 x 3 register tiles of the 256 threads.
            // Measured on the 24^3x48 setup: CH = 2 (4 CTAs per SM) 0.73 s, 1: 0.76, 4: 0.76, 8: 0.89;
            // WD_ASM_CH = 1, 2, 4, 8 overrides
            int ch = 2;
            if (const char *e = getenv("WD_ASM_CH")) ch = atoi(e) == 1 ? 1 : atoi(e) == 4 ? 4 : atoi(e) == 8 ? 8 : 2;
#define WD_ASM_CASE(CH)                                                                                          \
            if (ch == CH) {                                                                                      \
                const size_t smem2 = sizeof(cdd) * 3 * CH * 12 * (size_t)ncd;                                     \
                WD_CUDA(cudaFuncSetAttribute(k_assemble_dd2<CH>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                             (int)smem2));                                                        \
                k_assemble_dd2<CH><<<5 * g->Vc, 256, smem2, c->st>>>(g->Phi, g->Plo, (const double2 *)ulex, bc,   \
                                                                     c->kappa, g->Dc, M);                         \
            }
            WD_ASM_CASE(1) WD_ASM_CASE(2) WD_ASM_CASE(4) WD_ASM_CASE(8)
#undef WD_ASM_CASE
        } else {
            WD_CUDA(cudaFuncSetAttribute(k_assemble_dd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_assemble_dd<<<5 * g->Vc, 256, smem, c->st>>>(g->Phi, g->Plo, (const double2 *)ulex, bc, c->kappa, g->Dc,
                                                           M);
        }
    } else {
        WD_CUDA(cudaFuncSetAttribute(k_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_assemble<<<5 * g->Vc, 256, smem, c->st>>>(g->P, (const double2 *)ulex, bc, c->kappa, g->Dc, M);
    }
    k_dc_backward<<<1184, 256, 0, c->st>>>(g->Dc, g->nbr, g->Vc, ncd, nv);
    phase("Galerkin assembly");
    k_dc_to32<<<1184, 256, 0, c->st>>>(g->Dc, g->Dc32, g->Dclo, (long)nD);
    k_dc_to32<<<1184, 256, 0, c->st>>>(g->Gt, g->Ghi, g->Glo, (long)g->Vc * agg[3] * 2 * nv * nv);
    c->launches += 9;
    WD_CUDA(cudaGetLastError());
    WD_TRY(coarse_tc_build(c));
    WD_CUDA(cudaStreamSynchronize(c->st));
    phase("coarse copies, TC operand");
    return WD_OK;
}

extern "C" int wd_coarse_apply(wd_ctx *c, const double *in, double *out, int nrhs, int prec) {
    if (!c || !c->mg) { set_error("wd_coarse_apply: call wd_mg_setup first"); return WD_EINVAL; }
    if (nrhs < 0 || ((!in || !out) && nrhs > 0) || prec < 0 || prec > 2) { set_error("wd_coarse_apply: bad argument"); return WD_EINVAL; }
    if (nrhs == 0) return WD_OK;
    if (prec == P64) return coarse_apply64(c, in, out, nullptr, 0.0, 1.0, nrhs);
    const Space sp = coarse_space(c);
    // WD_MIXED_FP32: BF16-pair operands, WD_MIXED_BF16: BF16 operands on the
    // tensor cores; the FP32 blocks on the CUDA cores where those are unavailable
    // (WD_COARSE_FP32=1 forces the FP32 CUDA-core blocks, for tests)
    const char *f32 = getenv("WD_COARSE_FP32");
    const bool tc = coarse_tc_ok(c) && (prec == P16 || c->mg->Wlo) && !(f32 && atoi(f32) > 0);
    void *xl, *yl;
    WD_TRY(ws_get(c, "ca.x", space_bytes(sp, P32, nrhs), &xl));
    WD_TRY(ws_get(c, "ca.y", space_bytes(sp, P32, nrhs), &yl));
    WD_TRY(blas_copy_convert(c, sp, P64, in, P32, xl, nrhs, nullptr));
    if (tc) WD_TRY(coarse_tc_apply(c, xl, (float *)yl, nrhs, prec == P32));
    else WD_TRY(coarse_apply32(c, (const float *)xl, (float *)yl, nrhs));
    WD_TRY(blas_copy_convert(c, sp, P32, yl, P64, out, nrhs, nullptr));
    if (tc) WD_TRY(coarse_tc_check(c));
    return WD_OK;
}

extern "C" int wd_restrict(wd_ctx *c, const double *fine, double *coarse, int nrhs) {
    if (!c || !c->mg) { set_error("wd_restrict: call wd_mg_setup first"); return WD_EINVAL; }
    if (nrhs <= 0) return nrhs == 0 ? WD_OK : WD_EINVAL;
    const size_t f = field_bytes(c->g, P64, nrhs);
    double *e, *o;
    WD_TRY(ws_get(c, "rp.e", f, (void **)&e));
    WD_TRY(ws_get(c, "rp.o", f, (void **)&o));
    WD_TRY(user_to_eo(c, fine, true, P64, e, o, nrhs));
    return mg_restrict_eo(c, e, o, coarse, nrhs);
}

extern "C" int wd_prolong(wd_ctx *c, const double *coarse, double *fine, int nrhs) {
    if (!c || !c->mg) { set_error("wd_prolong: call wd_mg_setup first"); return WD_EINVAL; }
    if (nrhs <= 0) return nrhs == 0 ? WD_OK : WD_EINVAL;
    const size_t f = field_bytes(c->g, P64, nrhs);
    double *e, *o;
    WD_TRY(ws_get(c, "rp.e", f, (void **)&e));
    WD_TRY(ws_get(c, "rp.o", f, (void **)&o));
    WD_TRY(mg_prolong_eo(c, coarse, e, o, nrhs));
    return eo_to_user(c, e, o, P64, fine, true, nrhs);
}

extern "C" int wd_coarse_solve(wd_ctx *c, const double *b, double *x, int nrhs, double tol, int prec, int max_iter,
                               double *true_resid_out) {
    if (!c || !c->mg) { set_error("wd_coarse_solve: call wd_mg_setup first"); return WD_EINVAL; }
    if (nrhs < 0 || ((!b || !x) && nrhs > 0) || !(tol > 0) || max_iter < 1 || prec < 0 || prec > 2) {
        set_error("wd_coarse_solve: bad argument");
        return WD_EINVAL;
    }
    if (nrhs == 0) return WD_OK;
    int s = coarse_solve(c, b, x, nrhs, tol, prec, max_iter, true_resid_out);
    WD_CUDA(cudaStreamSynchronize(c->st));
    return s;
}
