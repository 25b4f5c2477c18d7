// Batched solves over lattices of different sizes.
//
// A wd_batch groups contexts (one gauge field each, any even extents) that
// share a CUDA stream.  wd_batch_solve runs their mixed-precision solves in
// lockstep: every inner BiCGStab iteration applies the even-odd Schur operator
// of all lattices with two persistent batched stencil launches (one work list
// over every lattice's site and RHS tiles) instead of two launches per
// lattice, and the Krylov BLAS of each lattice follows.  With use_graph the
// inner iterations between convergence checks are captured once into a CUDA
// graph and replayed, so the host issues one graph launch per check instead of
// ~(4 + 8 L) kernel launches per iteration.  The FP64 outer loop (defect
// correction) is per lattice, as in wd_solve.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <string>
#include <vector>

#include "wd_internal.h"

struct wd_batch {
    std::vector<wd_ctx *> c;
    cudaStream_t st;      // the contexts' stream
    cudaStream_t priv;    // private non-blocking stream the solves run on (capturable)
    cudaEvent_t ev;
};

namespace wd {

struct Lat {
    wd_ctx *c;
    int nrhs;
    double *be, *bo, *xe, *xo, *bhat, *r64, *tmp64, *blo, *scale, *rn2;
    void *tmplo;
    BiVecs V;
    std::vector<double> bnorm2, hsc, last;
    std::vector<int> iters;
    bool open;
};

static const void *gauge_par(wd_ctx *c, int prec, int p) {
    const size_t per = (size_t)8 * 9 * c->g.Vh * (prec == P64 ? 16 : prec == P32 ? 8 : 4);
    return (const char *)c->gauge[prec] + p * per;
}

// out_l = D_hat in_l for every lattice (inputs pp, outputs pw=FP32), two batched launches
static int batched_schur(std::vector<Lat> &L, int pp, bool which_s) {
    HopBatch B1, B2;
    B1.njobs = B2.njobs = (int)L.size();
    for (size_t j = 0; j < L.size(); ++j) {
        Lat &l = L[j];
        const void *in = which_s ? l.V.s : l.V.p;
        void *out = which_s ? l.V.t : l.V.v;
        HopArgs &a = B1.job[j];
        a.out = l.tmplo; a.in = in; a.w = nullptr; a.w2 = nullptr; a.a = 0.0; a.b = 1.0; a.c = 0.0;
        a.p = 1; a.nrhs = l.nrhs; a.nrb = 1; a.g = l.c->g; a.gauge = gauge_par(l.c, pp, 1);
        HopArgs &b = B2.job[j];
        b.out = out; b.in = l.tmplo; b.w = in; b.w2 = nullptr; b.a = 1.0; b.b = -l.c->kappa * l.c->kappa; b.c = 0.0;
        b.p = 0; b.nrhs = l.nrhs; b.nrb = 1; b.g = l.c->g; b.gauge = gauge_par(l.c, pp, 0);
    }
    cudaStream_t st = L[0].c->st;
    cudaError_t e;
    if (pp == P32) {
        e = launch_hop_batched<float, float, float, float>(B1, 2, st);
        if (e == cudaSuccess) e = launch_hop_batched<float, float, float, float>(B2, 2, st);
    } else {
        e = launch_hop_batched<bf16, bf16, bf16, bf16>(B1, 2, st);
        if (e == cudaSuccess) e = launch_hop_batched<bf16, float, bf16, bf16>(B2, 2, st);
    }
    L[0].c->launches += 2;
    if (e != cudaSuccess) { set_error("batched stencil: %s", cudaGetErrorString(e)); return WD_ECUDA; }
    return WD_OK;
}

static int iter_multi(std::vector<Lat> &L, int pp, int k) {
    for (int i = 0; i < k; ++i) {
        WD_TRY(batched_schur(L, pp, false));
        for (auto &l : L) WD_TRY(bicg_after_v(l.c, P32, pp, l.V, l.nrhs));
        WD_TRY(batched_schur(L, pp, true));
        for (auto &l : L) WD_TRY(bicg_after_t(l.c, P32, pp, l.V, l.nrhs));
    }
    return WD_OK;
}

static int active_total(std::vector<Lat> &L, int *hc) {
    for (size_t j = 0; j < L.size(); ++j)
        WD_CUDA(cudaMemcpyAsync(hc + j, L[j].V.count, sizeof(int), cudaMemcpyDeviceToHost, L[j].c->st));
    WD_CUDA(cudaStreamSynchronize(L[0].c->st));
    int a = 0;
    for (size_t j = 0; j < L.size(); ++j) a += hc[j];
    return a;
}

}  // namespace wd

using namespace wd;

extern "C" int wd_batch_create(wd_batch **out, wd_ctx *const *ctxs, int n) {
    if (!out || !ctxs || n < 1 || n > WD_MAX_BATCH) { set_error("wd_batch_create: 1..%d contexts", WD_MAX_BATCH); return WD_EINVAL; }
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) { set_error("wd_batch_create: null context"); return WD_EINVAL; }
        if (ctxs[i]->st != ctxs[0]->st) { set_error("wd_batch_create: contexts must share one stream"); return WD_EINVAL; }
    }
    wd_batch *b = new wd_batch();
    b->c.assign(ctxs, ctxs + n);
    b->st = ctxs[0]->st;
    if (cudaStreamCreateWithFlags(&b->priv, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        set_error("wd_batch_create: stream creation failed");
        return WD_ECUDA;
    }
    *out = b;
    return WD_OK;
}

extern "C" int wd_batch_destroy(wd_batch *b) {
    if (!b) return WD_OK;
    cudaStreamSynchronize(b->priv);
    cudaStreamDestroy(b->priv);
    cudaEventDestroy(b->ev);
    delete b;
    return WD_OK;
}

static int batch_solve_impl(wd_batch *b, cudaStream_t bst, const double *const *rhs, double *const *x,
                            const int *nrhs, double tol, int prec, int max_iter, int use_graph, int *iters_out,
                            double *resid_out);

// The solve runs on the batch's private stream (a CUDA graph cannot be captured
// on the legacy default stream), ordered after prior work of the contexts'
// stream and before later work on it.
extern "C" int wd_batch_solve(wd_batch *b, const double *const *rhs, double *const *x, const int *nrhs, double tol,
                              int prec, int max_iter, int use_graph, int *iters_out, double *resid_out) {
    if (!b) { set_error("wd_batch_solve: null batch"); return WD_EINVAL; }
    WD_CUDA(cudaEventRecord(b->ev, b->st));
    WD_CUDA(cudaStreamWaitEvent(b->priv, b->ev, 0));
    for (auto *c : b->c) c->st = b->priv;
    const int s = batch_solve_impl(b, b->priv, rhs, x, nrhs, tol, prec, max_iter, use_graph, iters_out, resid_out);
    cudaEventRecord(b->ev, b->priv);
    cudaStreamWaitEvent(b->st, b->ev, 0);
    for (auto *c : b->c) c->st = b->st;
    return s;
}

static int batch_solve_impl(wd_batch *b, cudaStream_t bst, const double *const *rhs, double *const *x,
                            const int *nrhs, double tol, int prec, int max_iter, int use_graph, int *iters_out,
                            double *resid_out) {
    if (!b || !rhs || !x || !nrhs || !(tol > 0) || max_iter < 1 || (prec != P32 && prec != P16)) {
        set_error("wd_batch_solve: bad argument (prec must be WD_MIXED_FP32 or WD_MIXED_BF16)");
        return WD_EINVAL;
    }
    const int n = (int)b->c.size();
    const int pp = prec;
    // stencil of the FP64 steps, as in solve_eo
    auto outer_of = [tol](wd_ctx *cc) { return tol < 1e-12 ? (int)P64 : cc->outer; };
    std::vector<Lat> L(n);
    for (int j = 0; j < n; ++j) {
        Lat &l = L[j];
        l.c = b->c[j];
        l.nrhs = nrhs[j];
        if (l.nrhs < 1 || !rhs[j] || !x[j]) { set_error("wd_batch_solve: lattice %d has no right-hand sides", j); return WD_EINVAL; }
        wd_ctx *c = l.c;
        const size_t f = field_bytes(c->g, P64, l.nrhs);
        WD_TRY(ws_get(c, "bt.be", f, (void **)&l.be));
        WD_TRY(ws_get(c, "bt.bo", f, (void **)&l.bo));
        WD_TRY(ws_get(c, "bt.xe", f, (void **)&l.xe));
        WD_TRY(ws_get(c, "bt.xo", f, (void **)&l.xo));
        WD_TRY(ws_get(c, "bt.bhat", f, (void **)&l.bhat));
        WD_TRY(ws_get(c, "bt.r64", f, (void **)&l.r64));
        WD_TRY(ws_get(c, "bt.tmp64", f, (void **)&l.tmp64));
        WD_TRY(ws_get(c, "bt.blo", field_bytes(c->g, P32, l.nrhs), (void **)&l.blo));
        WD_TRY(ws_get(c, "bt.tmplo", field_bytes(c->g, pp, l.nrhs), &l.tmplo));
        WD_TRY(ws_get(c, "bt.scale", sizeof(double) * 2 * l.nrhs, (void **)&l.scale));
        WD_TRY(ws_get(c, "bt.rn2", sizeof(double) * 2 * l.nrhs, (void **)&l.rn2));
        WD_TRY(alloc_bivecs(c, fine_space(c->g), P32, pp, l.nrhs, l.V, "bt.bi"));
        WD_TRY(user_to_eo(c, rhs[j], true, P64, l.be, l.bo, l.nrhs));
        const Space sp = fine_space(c->g);
        WD_TRY(blas_norm2(c, sp, P64, l.be, l.nrhs, l.rn2));
        WD_TRY(blas_norm2(c, sp, P64, l.bo, l.nrhs, l.rn2 + l.nrhs));
        std::vector<double> h(2 * l.nrhs);
        WD_CUDA(cudaMemcpyAsync(h.data(), l.rn2, sizeof(double) * 2 * l.nrhs, cudaMemcpyDeviceToHost, c->st));
        WD_CUDA(cudaStreamSynchronize(c->st));
        l.bnorm2.resize(l.nrhs);
        for (int r = 0; r < l.nrhs; ++r) l.bnorm2[r] = h[r] + h[l.nrhs + r];
        l.hsc.assign(2 * l.nrhs, 0.0);
        l.last.assign(l.nrhs, 0.0);
        l.iters.assign(l.nrhs, 0);
        // b_hat = b_e + k H_eo b_o; x = 0; r = b_hat
        WD_TRY(hop(c, outer_of(c), outer_of(c), 0, l.bhat, l.bo, l.be, 1.0, c->kappa, l.nrhs));
        WD_TRY(blas_zero(c, l.xe, f));
        WD_CUDA(cudaMemcpyAsync(l.r64, l.bhat, f, cudaMemcpyDeviceToDevice, c->st));
    }
    const bool graph = use_graph && !L[0].c->prof;
    const bool verbose = getenv("WD_VERBOSE") != nullptr;
    std::vector<int> hc(n);
    cudaGraphExec_t exec = nullptr;
    const int K = 4;
    int used = 0, status = WD_OK;
    for (int outer = 0; outer < 64; ++outer) {
        int open = 0;
        for (auto &l : L) {
            const Space sp = fine_space(l.c->g);
            WD_TRY(blas_norm2(l.c, sp, P64, l.r64, l.nrhs, l.rn2));
            WD_CUDA(cudaMemcpyAsync(l.last.data(), l.rn2, sizeof(double) * l.nrhs, cudaMemcpyDeviceToHost, l.c->st));
        }
        WD_CUDA(cudaStreamSynchronize(bst));
        for (auto &l : L) {
            l.open = false;
            for (int r = 0; r < l.nrhs; ++r) {
                const double rr = l.last[r];
                const bool done = !(rr > tol * tol * l.bnorm2[r]) || l.bnorm2[r] == 0.0;
                if (!isfinite(rr)) status = WD_EBREAKDOWN;
                l.hsc[r] = done || !isfinite(rr) ? 0.0 : 1.0 / sqrt(rr);
                l.hsc[l.nrhs + r] = done || !isfinite(rr) ? 0.0 : sqrt(rr);
                l.open = l.open || l.hsc[r] != 0.0;
            }
            open += l.open;
        }
        if (verbose) fprintf(stderr, "[wd] batch outer %d: %d lattices open, inner iterations %d\n", outer, open, used);
        if (open == 0 || used >= max_iter) break;
        for (auto &l : L) {
            const Space sp = fine_space(l.c->g);
            WD_CUDA(cudaMemcpyAsync(l.scale, l.hsc.data(), sizeof(double) * 2 * l.nrhs, cudaMemcpyHostToDevice, l.c->st));
            WD_TRY(blas_copy_convert(l.c, sp, P64, l.r64, P32, l.blo, l.nrhs, l.scale));
            WD_TRY(bicg_init(l.c, P32, pp, l.V, l.blo, l.nrhs, prec == P32 ? 1e-5 : 1e-2, nullptr));
        }
        // inner iterations in lockstep; K at a time, from a captured graph when allowed
        int active = active_total(L, hc.data());
        while (active > 0 && used < max_iter) {
            if (graph) {
                if (!exec) {
                    cudaGraph_t g;
                    WD_CUDA(cudaStreamBeginCapture(bst, cudaStreamCaptureModeThreadLocal));
                    int s = iter_multi(L, pp, K);
                    cudaError_t e = cudaStreamEndCapture(bst, &g);
                    if (s != WD_OK) return s;
                    WD_CUDA(e);
                    WD_CUDA(cudaGraphInstantiate(&exec, g, 0));
                    cudaGraphDestroy(g);
                }
                WD_CUDA(cudaGraphLaunch(exec, bst));
                L[0].c->launches += 1;
            } else {
                WD_TRY(iter_multi(L, pp, K));
            }
            used += K;
            active = active_total(L, hc.data());
        }
        for (auto &l : L) {
            std::vector<BiState> hs(l.nrhs);
            WD_CUDA(cudaMemcpyAsync(hs.data(), l.V.st, sizeof(BiState) * l.nrhs, cudaMemcpyDeviceToHost, l.c->st));
            WD_CUDA(cudaStreamSynchronize(l.c->st));
            for (int r = 0; r < l.nrhs; ++r) l.iters[r] += hs[r].iters;
            const Space sp = fine_space(l.c->g);
            WD_TRY(blas_axpy_mixed(l.c, sp, l.xe, P32, l.V.x, l.scale + l.nrhs, l.nrhs));
            // r = b_hat - D_hat x on FP64 fields (double-float stencil unless WD_DD=0 or tol < 1e-12)
            const int od = outer_of(l.c), ot = od == PDD ? PDDL : od;
            WD_TRY(hop(l.c, od, ot, 1, l.tmp64, l.xe, nullptr, 0.0, 1.0, l.nrhs));
            WD_TRY(hop(l.c, ot, od, 0, l.r64, l.tmp64, l.bhat, 1.0, l.c->kappa * l.c->kappa, l.nrhs, false, l.xe, -1.0));
        }
    }
    if (exec) cudaGraphExecDestroy(exec);
    int ri = 0;
    for (int j = 0; j < n; ++j) {
        Lat &l = L[j];
        WD_TRY(hop(l.c, outer_of(l.c), outer_of(l.c), 1, l.xo, l.xe, l.bo, 1.0, l.c->kappa, l.nrhs));
        WD_TRY(eo_to_user(l.c, l.xe, l.xo, P64, x[j], true, l.nrhs));
        int mx = 0;
        for (int r = 0; r < l.nrhs; ++r) {
            mx = l.iters[r] > mx ? l.iters[r] : mx;
            if (status == WD_OK && l.bnorm2[r] > 0 && !(l.last[r] <= tol * tol * l.bnorm2[r])) status = WD_ENOCONV;
            if (resid_out) resid_out[ri + r] = l.bnorm2[r] > 0 ? sqrt(l.last[r] / l.bnorm2[r]) : 0.0;
        }
        ri += l.nrhs;
        if (iters_out) iters_out[j] = mx;
    }
    WD_CUDA(cudaStreamSynchronize(bst));
    if (status != WD_OK) set_error("wd_batch_solve: %s", status == WD_ENOCONV ? "not converged" : "breakdown");
    return status;
}
