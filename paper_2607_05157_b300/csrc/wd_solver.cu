// Even-odd preconditioned multi-RHS solves with FP64 defect correction.
//
// With D = [[1, -k H_eo], [-k H_oe, 1]] (even sites first), the even-site
// Schur complement is  D_hat = 1 - k^2 H_eo H_oe,  and
//   D_hat x_e = b_e + k H_eo b_o,   x_o = b_o + k H_oe x_e
// solve D x = b exactly; the full residual of x equals the Schur residual on
// the even sites.  The Krylov solver is BiCGStab with per-RHS FP64 scalars
// (the paper names no method: Sec. 1 only needs the products D^{-1} eta).
//
// Mixed precision: the FP64 residual r = b_hat - D_hat x is
// normalised per RHS, solved to a loose relative tolerance in FP32 (or BF16
// storage with FP32 arithmetic), and the correction is added to x in FP64;
// repeated until the FP64 residual meets the requested tolerance.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <functional>
#include <string>
#include <algorithm>
#include <vector>

#include "wd_internal.h"

namespace wd {

int alloc_bivecs(wd_ctx *c, const Space &sp, int pw, int pp, int nrhs, BiVecs &V, const std::string &t) {
    const size_t fw = space_bytes(sp, pw, nrhs), fp = space_bytes(sp, pp, nrhs);
    WD_TRY(ws_get(c, (t + ".x").c_str(), fw, &V.x));
    WD_TRY(ws_get(c, (t + ".r").c_str(), fw, &V.r));
    WD_TRY(ws_get(c, (t + ".rh").c_str(), fw, &V.rh));
    WD_TRY(ws_get(c, (t + ".v").c_str(), fw, &V.v));
    WD_TRY(ws_get(c, (t + ".t").c_str(), fw, &V.t));
    WD_TRY(ws_get(c, (t + ".p").c_str(), fp, &V.p));
    WD_TRY(ws_get(c, (t + ".s").c_str(), fp, &V.s));
    WD_TRY(ws_get(c, (t + ".st").c_str(), sizeof(BiState) * nrhs, (void **)&V.st));
    V.sp = sp;
    V.bpr = reduction_bpr(sp.units, nrhs);
    WD_TRY(ws_get(c, (t + ".part").c_str(), sizeof(double) * 3 * V.bpr * nrhs, (void **)&V.part));
    WD_TRY(ws_get(c, (t + ".count").c_str(), sizeof(int), (void **)&V.count));
    WD_TRY(ws_get(c, (t + ".alist").c_str(), sizeof(int) * (size_t)nrhs, (void **)&V.alist));
    return WD_OK;
}

// ---- the BiCGStab loop on the device: a CUDA graph with a while node ------
// The body is two iterations (every kernel skips converged RHS) and a one-
// thread kernel that counts them and keeps the loop going while some RHS is
// active and the iteration limit is not reached.  The host launches the graph
// once per inner solve and reads the count back once; no launch latency and
// no host round trip per iteration.  The loop always ends: the count grows by
// two per body and the limit is finite.
__global__ void k_bicg_while(cudaGraphConditionalHandle h, const int *count, int *loop) {
    const int it = loop[0] + 2;
    loop[0] = it;
    cudaGraphSetConditional(h, (*count > 0 && it + 2 <= loop[1]) ? 1u : 0u);
}

static std::vector<uintptr_t> loop_key(wd_ctx *c, int pw, int pp, const BiVecs &V, int nrhs) {
    uint64_t kb;
    memcpy(&kb, &c->kappa, sizeof(kb));
    const char *ov = getenv("WD_HOP_R");
    return {(uintptr_t)V.x, (uintptr_t)V.r, (uintptr_t)V.rh, (uintptr_t)V.v, (uintptr_t)V.t, (uintptr_t)V.p,
            (uintptr_t)V.s, (uintptr_t)V.st, (uintptr_t)V.part, (uintptr_t)V.count, (uintptr_t)V.alist, (uintptr_t)V.op,
            V.sig[0], V.sig[1], V.sig[2], (uintptr_t)nrhs, (uintptr_t)pw, (uintptr_t)pp, (uintptr_t)V.bpr,
            (uintptr_t)V.sp.units, (uintptr_t)kb, (uintptr_t)std::hash<std::string>()(ov ? ov : "")};
}

static void loop_graph_free(wd_loop_graph &L) {
    if (L.exec) cudaGraphExecDestroy(L.exec);
    if (L.graph) cudaGraphDestroy(L.graph);
    L.exec = nullptr;
    L.graph = nullptr;
}

void wd_loops_free(wd_ctx *c) {
    for (auto &L : c->loops) loop_graph_free(L);
    c->loops.clear();
    if (c->gst) cudaStreamDestroy(c->gst);
    if (c->loop_dev) cudaFree(c->loop_dev);
    c->gst = nullptr;
    c->loop_dev = nullptr;
}

// Capture two iterations of V's loop into a while-node graph.  Returns false
// (and switches graphs off for this context) if the runtime refuses any step.
static bool loop_graph_build(wd_ctx *c, int pw, int pp, BiVecs &V, int nrhs, wd_loop_graph &L) {
    L.graph = nullptr;
    L.exec = nullptr;
    bool ok = true;
    if (!c->gst) ok = cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking) == cudaSuccess;
    if (ok && !c->loop_dev) ok = cudaMalloc(&c->loop_dev, 2 * sizeof(int)) == cudaSuccess;
    cudaGraphConditionalHandle h = 0;
    cudaGraph_t body = nullptr;
    if (ok) ok = cudaGraphCreate(&L.graph, 0) == cudaSuccess;
    if (ok) ok = cudaGraphConditionalHandleCreate(&h, L.graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
    if (ok) {
        cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        ok = cudaGraphAddNode(&node, L.graph, nullptr, nullptr, 0, &np) == cudaSuccess;
        if (ok) body = np.conditional.phGraph_out[0];
    }
    if (ok) ok = cudaStreamBeginCaptureToGraph(c->gst, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) ==
                 cudaSuccess;
    if (ok) {
        cudaStream_t saved = c->st;
        const int64_t l0 = c->launches;
        c->st = c->gst;
        int s = bicg_iter(c, pw, pp, V, nrhs);
        if (s == WD_OK) s = bicg_iter(c, pw, pp, V, nrhs);
        if (s == WD_OK) k_bicg_while<<<1, 1, 0, c->gst>>>(h, V.count, c->loop_dev);
        c->st = saved;
        L.kernels = (int)(c->launches - l0) + 1;
        c->launches = l0;                 // captured, not run
        cudaGraph_t out = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->gst, &out);
        ok = s == WD_OK && e == cudaSuccess;
    }
    if (ok) ok = cudaGraphInstantiate(&L.exec, L.graph, 0) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        loop_graph_free(L);
        c->graph_off = true;
        if (getenv("WD_VERBOSE")) fprintf(stderr, "[wd] BiCGStab loop graph refused: plain loops from now on\n");
    }
    return ok;
}

// Run up to max_more iterations (an even number, >= 2) on the device; *done =
// iterations run.  *used = false if graphs are unavailable (nothing ran).
static int loop_graph_run(wd_ctx *c, int pw, int pp, BiVecs &V, int nrhs, int max_more, int *done, bool *used) {
    *used = false;
    *done = 0;
    const std::vector<uintptr_t> key = loop_key(c, pw, pp, V, nrhs);
    wd_loop_graph *L = nullptr;
    for (auto &g : c->loops)
        if (g.key == key) L = &g;
    if (!L) {
        wd_loop_graph G;
        if (!loop_graph_build(c, pw, pp, V, nrhs, G)) return WD_OK;
        G.key = key;
        if (c->loops.size() >= 16) {      // keep the cache small
            loop_graph_free(c->loops.front());
            c->loops.erase(c->loops.begin());
        }
        c->loops.push_back(G);
        L = &c->loops.back();
    }
    int *h;
    WD_TRY(hws_get(c, "loop", 2 * sizeof(int), (void **)&h));
    h[0] = 0;
    h[1] = max_more;
    WD_CUDA(cudaMemcpyAsync(c->loop_dev, h, 2 * sizeof(int), cudaMemcpyHostToDevice, c->st));
    WD_CUDA(cudaGraphLaunch(L->exec, c->st));
    WD_CUDA(cudaMemcpyAsync(h, c->loop_dev, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaStreamSynchronize(c->st));
    *done = h[0];
    *used = true;
    c->launches += (int64_t)L->kernels * (h[0] / 2) + 1;
    return WD_OK;
}

// Run BiCGStab iterations until no RHS is active or max_iter is reached.
// Every kernel of an iteration (stencil and BLAS) skips the RHS that have
// converged (the stencil walks the active-RHS list set here).  The first two
// iterations run as plain launches (they tune the stencil shapes and touch
// every workspace); the rest run inside a captured graph whose while node
// checks convergence on the device, or -- when profiling with per-launch
// events, with WD_NO_GRAPH set, or if the runtime refuses the graph -- as
// plain launches with the host reading the active count every second
// iteration.
static int bicg_run(wd_ctx *c, int pw, int pp, BiVecs &V, int nrhs, int max_iter, int *ran) {
    int *hcount;
    WD_TRY(hws_get(c, "count", sizeof(int), (void **)&hcount));
    int it = 0;
    WD_CUDA(cudaMemcpyAsync(hcount, V.count, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaStreamSynchronize(c->st));
    int active = *hcount;
    struct MaskGuard {
        wd_ctx *c;
        ~MaskGuard() { c->alist = nullptr; c->acount = nullptr; c->act_count = -1; }
    } guard{c};
    c->alist = V.alist;
    c->acount = V.count;
    c->act_count = active;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->st, &cs);
    const bool graphs = V.graph_ok && !c->prof && !c->graph_off && cs == cudaStreamCaptureStatusNone &&
                        getenv("WD_NO_GRAPH") == nullptr;
    // profiling: check after every iteration, so that the stencil's recorded
    // bytes count exactly the RHS that still work
    const int check = c->prof ? 1 : 2;
    while (active > 0 && it < max_iter) {
        if (graphs && it >= 2 && max_iter - it >= 2 && !c->graph_off) {
            int done = 0;
            bool used = false;
            WD_TRY(loop_graph_run(c, pw, pp, V, nrhs, (max_iter - it) & ~1, &done, &used));
            if (used) {
                it += done;
                WD_CUDA(cudaMemcpyAsync(hcount, V.count, sizeof(int), cudaMemcpyDeviceToHost, c->st));
                WD_CUDA(cudaStreamSynchronize(c->st));
                active = *hcount;
                continue;
            }
        }
        int k = check < max_iter - it ? check : max_iter - it;
        for (int i = 0; i < k; ++i) WD_TRY(bicg_iter(c, pw, pp, V, nrhs));
        it += k;
        WD_CUDA(cudaMemcpyAsync(hcount, V.count, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        WD_CUDA(cudaStreamSynchronize(c->st));
        active = *hcount;
        c->act_count = active;
    }
    *ran = it;
    return WD_OK;
}

static int read_states(wd_ctx *c, const BiState *dst, int nrhs, std::vector<BiState> &h) {
    h.resize(nrhs);
    WD_CUDA(cudaMemcpyAsync(h.data(), dst, sizeof(BiState) * nrhs, cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaStreamSynchronize(c->st));
    return WD_OK;
}

int dc_solve(wd_ctx *c, const Problem &P, const double *b, double *x, int nrhs, const double *bnorm2_dev,
             const std::vector<double> &bnorm2, double tol, int prec, int max_iter, std::vector<int> &iters,
             std::vector<double> &last_rn2) {
    const size_t f64 = space_bytes(P.sp, P64, nrhs);
    const std::string tag(P.tag);
    const bool verbose = getenv("WD_VERBOSE") != nullptr;
    iters.assign(nrhs, 0);
    last_rn2.assign(nrhs, 0.0);
    int status = WD_OK;
    if (prec == P64) {
        BiVecs V;
        WD_TRY(alloc_bivecs(c, P.sp, P64, P64, nrhs, V, tag + ".bi64"));
        V.op = P.op64;
        V.op_user = P.u64;
        V.graph_ok = P.graph_ok;
        for (int q = 0; q < 3; ++q) V.sig[q] = P.sig64[q];
        // the recursive residual drifts from the true one: aim at half the tolerance
        WD_TRY(bicg_init(c, P64, P64, V, b, nrhs, 0.5 * tol, bnorm2_dev));
        int ran = 0;
        WD_TRY(bicg_run(c, P64, P64, V, nrhs, max_iter, &ran));
        WD_CUDA(cudaMemcpyAsync(x, V.x, f64, cudaMemcpyDeviceToDevice, c->st));
        std::vector<BiState> hs;
        WD_TRY(read_states(c, V.st, nrhs, hs));
        for (int r = 0; r < nrhs; ++r) {
            iters[r] = hs[r].iters;
            last_rn2[r] = hs[r].rr;
            if (hs[r].flag) status = WD_EBREAKDOWN;
            else if (hs[r].rr > hs[r].thr && status == WD_OK) status = WD_ENOCONV;
        }
        return status;
    }
    const int pw = P32, pp = prec == P32 ? P32 : P16;
    const double inner_tol = P.inner_tol > 0.0 ? P.inner_tol : prec == P32 ? 1e-5 : 1e-2;
    BiVecs V;
    WD_TRY(alloc_bivecs(c, P.sp, pw, pp, nrhs, V, tag + (prec == P32 ? ".bi32" : ".bi16")));
    V.op = P.oplo;
    V.op_user = P.ulo;
    V.graph_ok = P.graph_ok;
    for (int q = 0; q < 3; ++q) V.sig[q] = P.siglo[q];
    double *r64, *scale_d, *rn2_d, *blo, *hsc;
    WD_TRY(ws_get(c, (tag + ".r64").c_str(), f64, (void **)&r64));
    WD_TRY(ws_get(c, (tag + ".blo").c_str(), space_bytes(P.sp, pw, nrhs), (void **)&blo));
    WD_TRY(ws_get(c, (tag + ".scale").c_str(), sizeof(double) * 3 * nrhs, (void **)&scale_d));
    WD_TRY(ws_get(c, (tag + ".rn2").c_str(), sizeof(double) * nrhs, (void **)&rn2_d));
    WD_TRY(hws_get(c, (tag + ".hscale").c_str(), sizeof(double) * 3 * nrhs, (void **)&hsc));
    const bool can_update = P.opupd != nullptr;
    std::vector<double> upd_acc(nrhs, 0.0);    // sum of the update error bounds, per RHS
    // the solution: FP64, or (x_ddl) a double-float layout copy updated in
    // double-float arithmetic and assembled into FP64 once at the end
    void *xd = nullptr;
    if (P.x_ddl) {
        WD_TRY(ws_get(c, (tag + ".xdd").c_str(), f64, &xd));
        WD_CUDA(cudaMemsetAsync(xd, 0, f64, c->st));
    } else {
        WD_TRY(blas_zero(c, x, f64));
    }
    // residual r64: FP64, or the double-float layout (same size) when the
    // problem's residual writes it
    const int rp = P.res_ddl ? PDDL : P64;
    if (P.res_ddl) {
        WD_CUDA(launch_to_ddl(b, r64, 12L * P.sp.units * nrhs, c->st));
        c->launches++;
    } else {
        WD_CUDA(cudaMemcpyAsync(r64, b, f64, cudaMemcpyDeviceToDevice, c->st));
    }
    std::vector<double> rn2(nrhs);
    int used = 0;
    for (int outer = 0; outer < 64; ++outer) {
        WD_TRY(blas_norm2(c, P.sp, rp, r64, nrhs, rn2_d));
        WD_CUDA(cudaMemcpyAsync(rn2.data(), rn2_d, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->st));
        WD_CUDA(cudaStreamSynchronize(c->st));
        int open = 0;
        double worst_rel = 0.0;
        for (int r = 0; r < nrhs; ++r) {
            const double rn = sqrt(rn2[r]) + upd_acc[r];
            const bool done = !(rn > tol * sqrt(bnorm2[r])) || bnorm2[r] == 0.0;
            if (!isfinite(rn2[r])) status = WD_EBREAKDOWN;
            hsc[r] = done || !isfinite(rn2[r]) ? 0.0 : 1.0 / sqrt(rn2[r]);
            hsc[nrhs + r] = done || !isfinite(rn2[r]) ? 0.0 : sqrt(rn2[r]);
            hsc[2 * nrhs + r] = -hsc[nrhs + r];
            open += hsc[r] != 0.0;
            if (hsc[r] != 0.0) worst_rel = fmax(worst_rel, sqrt(rn2[r] / bnorm2[r]));
        }
        // this step's residual by the recursive update (Problem::opupd)
        const bool recursive = can_update && isfinite(worst_rel) && P.upd_err * worst_rel <= 0.25 * tol;
        last_rn2 = rn2;
        if (verbose) {
            double worst = 0;
            for (int r = 0; r < nrhs; ++r)
                if (bnorm2[r] > 0) worst = fmax(worst, sqrt(rn2[r] / bnorm2[r]));
            fprintf(stderr, "[wd] %s outer %d: max rel residual %.3e, open %d, inner iterations so far %d\n",
                    P.tag, outer, worst, open, used);
        }
        if (open == 0 || used >= max_iter) break;
        WD_CUDA(cudaMemcpyAsync(scale_d, hsc, sizeof(double) * 3 * nrhs, cudaMemcpyHostToDevice, c->st));
        // b_lo = r / |r|   (zero for converged RHS, which then stay inactive)
        WD_TRY(blas_copy_convert(c, P.sp, rp, r64, pw, blo, nrhs, scale_d));
        WD_TRY(bicg_init(c, pw, pp, V, blo, nrhs, inner_tol, nullptr));
        int ran = 0;
        WD_TRY(bicg_run(c, pw, pp, V, nrhs, max_iter - used, &ran));
        used += ran;
        std::vector<BiState> hs;
        WD_TRY(read_states(c, V.st, nrhs, hs));
        for (int r = 0; r < nrhs; ++r) iters[r] += hs[r].iters;
        if (verbose) {
            int flags = 0, mx = 0;
            for (int r = 0; r < nrhs; ++r) { flags += hs[r].flag; mx = hs[r].iters > mx ? hs[r].iters : mx; }
            fprintf(stderr, "[wd]   inner: ran %d, max iters %d, breakdowns %d\n", ran, mx, flags);
        }
        // x += |r| e  (FP64 or double-float), then the FP64 residual r = b - A x,
        // or the recursive update r -= |r| A e once the residual is small
        if (P.x_ddl) WD_TRY(blas_axpy_ddl(c, P.sp, xd, V.x, scale_d + nrhs, nrhs));
        else WD_TRY(blas_axpy_mixed(c, P.sp, x, pw, V.x, scale_d + nrhs, nrhs));
        if (recursive) {
            // r -= |r| A e: A e is close to r / |r|, so an operator error of
            // upd_err relative to |r| is all the update adds
            void *y;
            WD_TRY(ws_get(c, (tag + ".upd").c_str(), space_bytes(P.sp, pw, nrhs), &y));
            WD_TRY(P.opupd(c, V.x, y, nrhs, P.uupd));
            if (P.res_ddl) WD_TRY(blas_axpy_ddl(c, P.sp, r64, y, scale_d + 2 * nrhs, nrhs));
            else WD_TRY(blas_axpy_mixed(c, P.sp, r64, pw, y, scale_d + 2 * nrhs, nrhs));
            for (int r = 0; r < nrhs; ++r) upd_acc[r] += P.upd_err * hsc[nrhs + r];
        } else {
            WD_TRY(P.res64(c, b, P.x_ddl ? (const double *)xd : x, r64, nrhs, P.ures));
            std::fill(upd_acc.begin(), upd_acc.end(), 0.0);
        }
        if (verbose) fprintf(stderr, "[wd]   residual by %s\n", recursive ? "recursive update" : "res64");
    }
    if (P.x_ddl) WD_TRY(blas_ddl_to_f64(c, P.sp, xd, x, nrhs));
    if (status == WD_OK)
        for (int r = 0; r < nrhs; ++r)
            if (bnorm2[r] > 0 && !(last_rn2[r] <= tol * tol * bnorm2[r])) status = WD_ENOCONV;
    return status;
}

// ---- the even-site Schur operator D_hat = 1 - k^2 H_eo H_oe ----------------
struct SchurArgs {
    int pin, pout;
    void *tmp;      // odd-parity field in precision pin
    bool x_ddl;     // schur_res64: x in the double-float layout
};

static int schur_op(wd_ctx *c, const void *in, void *out, int nrhs, void *u) {
    SchurArgs *S = (SchurArgs *)u;
    WD_TRY(hop(c, S->pin, S->pin, 1, S->tmp, in, nullptr, 0.0, 1.0, nrhs));
    return hop(c, S->pin, S->pout, 0, out, S->tmp, in, 1.0, -c->kappa * c->kappa, nrhs);
}

// r = b - D_hat x = b - x + k^2 H_eo H_oe x on FP64 fields, with the stencil
// S->pin (P64, or PDD: double-float arithmetic, the odd intermediate kept in
// the double-float layout); r in S->pout (P64, PDD = FP64, or PDDL)
static int schur_res64(wd_ctx *c, const double *b, const double *x, double *r, int nrhs, void *u) {
    SchurArgs *S = (SchurArgs *)u;
    const int pt = S->pin == PDD ? PDDL : S->pin;
    WD_TRY(hop(c, S->x_ddl ? PDDL : S->pin, pt, 1, S->tmp, x, nullptr, 0.0, 1.0, nrhs));
    return hop(c, pt, S->pout, 0, r, S->tmp, b, 1.0, c->kappa * c->kappa, nrhs, false, x, -1.0, nullptr, S->x_ddl);
}

// dst[rhs][i] = fac[rhs] * src[rhs][i] for FP64 eo fields (per = doubles per
// RHS of one parity); fac a power of two, so the product is exact
__global__ void k_scale_rhs(double *dst, const double *src, const double *fac, long per, int nrhs) {
    const long n = per * nrhs;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        dst[i] = fac[i / per] * src[i];
}

static int scale_rhs(wd_ctx *c, double *dst, const double *src, const double *fac, int nrhs) {
    k_scale_rhs<<<1184, 256, 0, c->st>>>(dst, src, fac, 24L * c->g.Vh, nrhs);
    c->launches++;
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

// The even-odd solve entirely in FP32, for loose targets (tol >= 1e-6: the
// multigrid setup's inverse iterations): FP32 copies of b, the Schur source
// b_hat = b_e + k H_eo b_o, BiCGStab on D_hat to half the target (its
// recursive residual), x_o = b_o + k H_oe x_e, both parities back to FP64.
// FP32 rounding moves the residual by ~1e-7 of |b|, an order below such a
// target, so no FP64 residual certifies it.
int solve_eo_fp32(wd_ctx *c, const double *b_e, const double *b_o, double *x_e, double *x_o, int nrhs, double tol) {
    if (nrhs <= 0) return WD_OK;
    if (tol < 1e-6) { set_error("solve_eo_fp32: tolerance below 1e-6"); return WD_EINVAL; }
    const Space sp = fine_space(c->g);
    const size_t f32 = field_bytes(c->g, P32, nrhs);
    void *be, *bo, *bh, *xo, *tmp;
    WD_TRY(ws_get(c, "s32.be", f32, &be));
    WD_TRY(ws_get(c, "s32.bo", f32, &bo));
    WD_TRY(ws_get(c, "s32.bh", f32, &bh));
    WD_TRY(ws_get(c, "s32.xo", f32, &xo));
    WD_TRY(ws_get(c, "s32.tmp", f32, &tmp));
    WD_TRY(blas_copy_convert(c, sp, P64, b_e, P32, be, nrhs, nullptr));
    WD_TRY(blas_copy_convert(c, sp, P64, b_o, P32, bo, nrhs, nullptr));
    WD_TRY(hop(c, P32, P32, 0, bh, bo, be, 1.0, c->kappa, nrhs));
    SchurArgs slo = {P32, P32, tmp, false};
    BiVecs V;
    WD_TRY(alloc_bivecs(c, sp, P32, P32, nrhs, V, "s32.bi"));
    V.op = schur_op;
    V.op_user = &slo;
    V.graph_ok = true;
    V.sig[0] = P32; V.sig[1] = P32; V.sig[2] = (uintptr_t)tmp;
    WD_TRY(bicg_init(c, P32, P32, V, bh, nrhs, 0.5 * tol, nullptr));
    int ran = 0;
    WD_TRY(bicg_run(c, P32, P32, V, nrhs, 100000, &ran));
    std::vector<BiState> hs;
    WD_TRY(read_states(c, V.st, nrhs, hs));
    int status = WD_OK;
    for (int r = 0; r < nrhs; ++r)
        if (hs[r].flag) status = WD_EBREAKDOWN;
    WD_TRY(hop(c, P32, P32, 1, xo, V.x, bo, 1.0, c->kappa, nrhs));
    WD_TRY(blas_copy_convert(c, sp, P32, V.x, P64, x_e, nrhs, nullptr));
    WD_TRY(blas_copy_convert(c, sp, P32, xo, P64, x_o, nrhs, nullptr));
    if (status != WD_OK) set_error("solve: breakdown");
    return status;
}

int solve_eo(wd_ctx *c, const double *b_e, const double *b_o, double *x_e, double *x_o, int nrhs, double tol,
             int prec, int max_iter, int *iters_out, double *resid_out, const int *src_tsup,
             const double **bhat_out) {
    if (nrhs <= 0) return WD_OK;
    if (!x_o && resid_out) { set_error("solve: the true residual needs the odd sites"); return WD_EINVAL; }
    const double k = c->kappa;
    const Space sp = fine_space(c->g);
    const size_t f64 = field_bytes(c->g, P64, nrhs);
    double *bhat, *bn2, *tmp64;
    WD_TRY(ws_get(c, "sol.bhat", f64, (void **)&bhat));
    WD_TRY(ws_get(c, "sol.tmp64", f64, (void **)&tmp64));
    WD_TRY(ws_get(c, "sol.bn2", sizeof(double) * 3 * nrhs, (void **)&bn2));
    // |b|^2 over both parities
    WD_TRY(blas_norm2(c, sp, P64, b_e, nrhs, bn2));
    WD_TRY(blas_norm2(c, sp, P64, b_o, nrhs, bn2 + nrhs));
    std::vector<double> bnorm2(2 * nrhs);
    WD_CUDA(cudaMemcpyAsync(bnorm2.data(), bn2, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaStreamSynchronize(c->st));
    for (int r = 0; r < nrhs; ++r) bnorm2[r] += bnorm2[nrhs + r];
    bnorm2.resize(nrhs);
    // The FP64 steps (source, residuals, reconstruction) of a mixed solve run
    // the double-float stencil: FP64 fields, ~2^-44 normwise, well below the
    // tolerances the outer loop certifies (tol < 1e-12 and the FP64 mode keep
    // FP64 arithmetic).
    const int pd = prec == P64 || tol < 1e-12 ? P64 : c->outer;
    // A double-float number holds magnitudes in [2^-103, 2^128): a source whose
    // norm lies outside [2^-30, 2^30] is solved as 2^-e b (e its binary
    // exponent, so the scaled norm lies in [1, 2)) and the solution scaled back
    // by 2^e.  Powers of two commute with every rounding on the way, so the
    // result is the unscaled solve's, scaled.
    std::vector<double> fac(nrhs, 1.0);
    bool rescale = false;
    if (pd == PDD)
        for (int r = 0; r < nrhs; ++r) {
            const double nb = sqrt(bnorm2[r]);
            if (nb > 0.0 && isfinite(nb) && (nb < 0x1p-30 || nb > 0x1p30)) {
                int e;
                frexp(nb, &e);
                fac[r] = ldexp(1.0, 1 - e);
                bnorm2[r] *= fac[r] * fac[r];
                rescale = true;
            }
        }
    double *fac_dev = nullptr;
    std::vector<double> both;      // factors and their inverses (alive until the copy has run)
    if (rescale) {
        double *bs;
        WD_TRY(ws_get(c, "sol.bscaled", 2 * f64, (void **)&bs));
        WD_TRY(ws_get(c, "sol.fac", sizeof(double) * 2 * nrhs, (void **)&fac_dev));
        both = fac;
        for (int r = 0; r < nrhs; ++r) both.push_back(1.0 / fac[r]);
        WD_CUDA(cudaMemcpyAsync(fac_dev, both.data(), sizeof(double) * 2 * nrhs, cudaMemcpyHostToDevice, c->st));
        WD_TRY(scale_rhs(c, bs, b_e, fac_dev, nrhs));
        WD_TRY(scale_rhs(c, bs + f64 / sizeof(double), b_o, fac_dev, nrhs));
        b_e = bs;
        b_o = bs + f64 / sizeof(double);
    }
    WD_CUDA(cudaMemcpyAsync(bn2 + 2 * nrhs, bnorm2.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, c->st));
    // b_hat = b_e + k H_eo b_o
    WD_TRY(hop(c, pd, pd, 0, bhat, b_o, b_e, 1.0, k, nrhs, false, nullptr, 0.0, src_tsup));
    if (bhat_out) *bhat_out = bhat;

    const int pp = prec == P16 ? P16 : (prec == P32 ? P32 : P64);
    void *tmplo = nullptr;
    if (prec != P64) WD_TRY(ws_get(c, "sol.tmplo", field_bytes(c->g, pp, nrhs), &tmplo));
    SchurArgs s64 = {P64, P64, tmp64, false}, slo = {pp, P32, tmplo, false},
              sres = {pd, pd == PDD ? PDDL : pd, tmp64, pd == PDD};
    Problem P;
    P.sp = sp;
    P.op64 = schur_op; P.u64 = &s64;
    P.oplo = schur_op; P.ulo = &slo;
    P.res64 = schur_res64; P.ures = &sres;
    P.res_ddl = sres.pout == PDDL;
    P.x_ddl = sres.x_ddl;
    P.tag = "fine";
    // a loose target (the multigrid setup's inverse iterations solve to 1e-6):
    // take the FP32 inner solve deeper, so that one outer step can reach it
    if (prec == P32 && tol >= 1e-6) P.inner_tol = 0.5 * tol;
    // once the residual is small, r <- r - D_hat e with the FP32 operator of
    // the inner solves instead of a double-float residual (two FP32 hops in
    // place of two double-float ones): its normwise error, a few 1e-7 of |e|
    // at the masses of interest, stays below 1.5e-6 of |r|
    if (prec == P32) { P.opupd = schur_op; P.uupd = &slo; P.upd_err = 1.5e-6; }
    // the Schur operator's launches see the precisions and the odd workspace
    P.graph_ok = true;
    P.sig64[0] = s64.pin; P.sig64[1] = s64.pout; P.sig64[2] = (uintptr_t)s64.tmp;
    P.siglo[0] = slo.pin; P.siglo[1] = slo.pout; P.siglo[2] = (uintptr_t)slo.tmp;
    std::vector<int> iters;
    std::vector<double> last_rn2;
    int status = dc_solve(c, P, bhat, x_e, nrhs, bn2 + 2 * nrhs, bnorm2, tol, prec, max_iter, iters, last_rn2);
    if (status != WD_OK && status != WD_ENOCONV && status != WD_EBREAKDOWN) return status;
    // x_o = b_o + k H_oe x_e
    if (x_o) WD_TRY(hop(c, pd, pd, 1, x_o, x_e, b_o, 1.0, k, nrhs));
    // True FP64 residual of the full system, when asked for.  Without it the
    // last FP64 Schur residual (mixed modes) or the FP64 recursion (FP64 mode)
    // certifies convergence: the full residual of (x_e, x_o) equals the Schur
    // residual on the even sites.
    if (resid_out) {
        double *re, *ro, *n2;
        WD_TRY(ws_get(c, "sol.re", f64, (void **)&re));
        WD_TRY(ws_get(c, "sol.ro", f64, (void **)&ro));
        WD_TRY(ws_get(c, "sol.n2", sizeof(double) * 2 * nrhs, (void **)&n2));
        WD_TRY(hop(c, P64, P64, 0, re, x_o, b_e, 1.0, k, nrhs, false, x_e, -1.0));
        WD_TRY(hop(c, P64, P64, 1, ro, x_e, b_o, 1.0, k, nrhs, false, x_o, -1.0));
        WD_TRY(blas_norm2(c, sp, P64, re, nrhs, n2));
        WD_TRY(blas_norm2(c, sp, P64, ro, nrhs, n2 + nrhs));
        std::vector<double> h(2 * nrhs);
        WD_CUDA(cudaMemcpyAsync(h.data(), n2, sizeof(double) * 2 * nrhs, cudaMemcpyDeviceToHost, c->st));
        WD_CUDA(cudaStreamSynchronize(c->st));
        status = status == WD_EBREAKDOWN ? status : WD_OK;
        for (int r = 0; r < nrhs; ++r) {
            const double res = bnorm2[r] > 0 ? sqrt((h[r] + h[nrhs + r]) / bnorm2[r]) : 0.0;
            resid_out[r] = res;
            if (!(res <= tol * 1.0000001) && status == WD_OK) status = isfinite(res) ? WD_ENOCONV : WD_EBREAKDOWN;
        }
    }
    if (rescale) {
        // back to the caller's scale (the relative residuals above are scale-free)
        WD_TRY(scale_rhs(c, x_e, x_e, fac_dev + nrhs, nrhs));
        if (x_o) WD_TRY(scale_rhs(c, x_o, x_o, fac_dev + nrhs, nrhs));
        if (bhat_out) WD_TRY(scale_rhs(c, bhat, bhat, fac_dev + nrhs, nrhs));
    }
    WD_TRY(hop_err_check(c));
    if (iters_out)
        for (int r = 0; r < nrhs; ++r) iters_out[r] = iters[r];
    if (status != WD_OK) set_error("solve: %s", status == WD_ENOCONV ? "not converged within max_iter" : "breakdown");
    return status;
}

}  // namespace wd
