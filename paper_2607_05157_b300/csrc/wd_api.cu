// C ABI entry points of libwd: context life cycle, gauge ingest,
// D / D^dag application and solves, workspaces, profiling.
#include <stdarg.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "wd_internal.h"

namespace wd {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int ws_get(wd_ctx *c, const char *name, size_t bytes, void **out) {
    auto it = c->bufs.find(name);
    if (it != c->bufs.end() && it->second.second >= bytes) { *out = it->second.first; return WD_OK; }
    if (it != c->bufs.end()) {
        WD_CUDA(cudaStreamSynchronize(c->st));
        cudaFree(it->second.first);
        c->bufs.erase(it);
    }
    void *p = nullptr;
    size_t nb = bytes > 0 ? bytes : 16;
    if (cudaMalloc(&p, nb) != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes for '%s' failed", nb, name);
        return WD_ENOMEM;
    }
    c->bufs[name] = std::make_pair(p, nb);
    *out = p;
    return WD_OK;
}

int hws_get(wd_ctx *c, const char *name, size_t bytes, void **out) {
    auto it = c->hbufs.find(name);
    if (it != c->hbufs.end() && it->second.second >= bytes) { *out = it->second.first; return WD_OK; }
    if (it != c->hbufs.end()) {
        WD_CUDA(cudaStreamSynchronize(c->st));
        cudaFreeHost(it->second.first);
        c->hbufs.erase(it);
    }
    void *p = nullptr;
    size_t nb = bytes > 0 ? bytes : 16;
    if (cudaMallocHost(&p, nb) != cudaSuccess) {
        cudaGetLastError();
        set_error("pinned host allocation of %zu bytes for '%s' failed", nb, name);
        return WD_ENOMEM;
    }
    c->hbufs[name] = std::make_pair(p, nb);
    *out = p;
    return WD_OK;
}

void prof_begin(wd_ctx *c, int k, double bytes, int *slot) {
    *slot = -1;
    if (!c->prof) return;
    wd_prof_rec r;
    if (c->event_pool.size() >= 2) {
        r.a = c->event_pool.back(); c->event_pool.pop_back();
        r.b = c->event_pool.back(); c->event_pool.pop_back();
    } else {
        cudaEventCreate(&r.a);
        cudaEventCreate(&r.b);
    }
    r.kernel = k;
    r.bytes = bytes;
    cudaEventRecord(r.a, c->st);
    c->recs.push_back(r);
    *slot = (int)c->recs.size() - 1;
}

void prof_end(wd_ctx *c, int slot) {
    if (slot < 0) return;
    cudaEventRecord(c->recs[slot].b, c->st);
}

static const void *gauge_parity(wd_ctx *c, int prec, int p) {
    const size_t per = (size_t)8 * 9 * c->g.Vh * (prec == P64 ? 16 : prec == P32 ? 8 : 4);
    return (const char *)c->gauge[prec] + p * per;
}

static cudaError_t launch_hop_any(int pin, int pout, const HopArgs &A, int R, bool dag, int th, cudaStream_t st) {
    if (is_dd(pin)) return launch_hop_dd(A, R, dag, th, pout == PDDL, st);
    if (pin == P64) return launch_hop<double, double, double, double>(A, R, dag, th, st);
    if (pin == P32) return launch_hop<float, float, float, float>(A, R, dag, th, st);
    if (pout == P16) return launch_hop<bf16, bf16, bf16, bf16>(A, R, dag, th, st);
    return launch_hop<bf16, float, bf16, bf16>(A, R, dag, th, st);
}

static int rhs_bucket(int nrhs) {
    int b = 1;
    while (b < nrhs && b < 4096) b <<= 1;
    return b;
}

// Autotuner: time every (RHS tile, block size) candidate on this launch's own
// buffers (the real launch follows and overwrites `out`), keep the fastest per
// (input precision, output precision, RHS bucket).  Not usable during stream
// capture: the caller must tune (one uncaptured call) before capturing.
static int tune_hop(wd_ctx *c, int pin, int pout, const HopArgs &A, bool dag, int *R, int *th) {
    // WD_HOP_R = "R" or "R:threads" overrides the FP32/BF16 launch shape (R code as
    // below; 128 threads unless given), for experiments, profiling and tests
    // WD_DD_R = "R[:threads]" does the same for the double-float stencil (R = 1, 2
    // scalar, 11, 12 packed)
    if (is_dd(pin)) {
        const char *ov = getenv("WD_DD_R");
        if (ov && atoi(ov) > 0) {
            *R = atoi(ov);
            const char *colon = strchr(ov, ':');
            *th = colon && atoi(colon + 1) > 0 ? atoi(colon + 1) : 128;
            return WD_OK;
        }
    }
    if (pin == P32 || pin == P16) {
        const char *ov = getenv("WD_HOP_R");
        if (ov && atoi(ov) > 0) {
            *R = atoi(ov);
            const char *colon = strchr(ov, ':');
            *th = colon && atoi(colon + 1) > 0 ? atoi(colon + 1) : 128;
            return WD_OK;
        }
    }
    const int key = (pin * 8 + pout) * 8192 + rhs_bucket(A.nrhs);
    auto it = c->tuned.find(key);
    if (it != c->tuned.end()) { *R = it->second.first; *th = it->second.second; return WD_OK; }
    *R = c->hop_R[pin];
    *th = c->hop_threads[pin];
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c->st, &cs);
    if (!c->autotune || cs != cudaStreamCaptureStatusNone) return WD_OK;
    // RHS tile R (1, 2, 4; +10 = software-pipelined FP32 variant) x block size
    // (21, 22, 24 = timeslices staged through shared memory; block size fixed by the kernel)
    // (31, 32 / 41, 42 = next-direction prefetch into L1 / L2)
    // (51, 52 = plain, site tile fastest in the block order; 62 = two RHS with
    // registers capped for 20 resident warps per SM; 63-65 = the same with the
    // RHS tiles in groups of 4, 8, 16)
    // (32-thread blocks: more blocks per SM for launches with few RHS)
    const int Rs[18] = {1, 2, 4, 11, 12, 21, 22, 24, 31, 32, 41, 42, 51, 52, 62, 63, 64, 65};
    const int Ts[4] = {32, 64, 128, 256};
    cudaEvent_t e0, e1;
    WD_CUDA(cudaEventCreate(&e0));
    WD_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int i = 0; i < 18; ++i)
        for (int j = 0; j < 4; ++j) {
            if (pin == P64 && Rs[i] > 2) continue;                   // FP64: R = 1, 2 only (R = 4 spills)
            if (is_dd(pin) && Rs[i] != 1 && Rs[i] != 2 && Rs[i] != 11 && Rs[i] != 12) continue;
            if (is_dd(pin) && Ts[j] > 128) continue;                 // double-float: at most 128 threads
            if (Rs[i] > 20 && Rs[i] < 30 && j > 0) continue;   // staged: one block size
            if (Rs[i] > 30 && pin != P32 && pin != P16) continue;
            {
                const cudaError_t e = launch_hop_any(pin, pout, A, Rs[i], dag, Ts[j], c->st);   // warm
                if (e == cudaErrorNotSupported) continue;    // variant does not apply to this shape
                WD_CUDA(e);
            }
            WD_CUDA(cudaEventRecord(e0, c->st));
            for (int k = 0; k < 3; ++k) WD_CUDA(launch_hop_any(pin, pout, A, Rs[i], dag, Ts[j], c->st));
            WD_CUDA(cudaEventRecord(e1, c->st));
            WD_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            WD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            c->launches += 4;
            if (ms < best) { best = ms; *R = Rs[i]; *th = Ts[j]; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tuned[key] = std::make_pair(*R, *th);
    if (getenv("WD_VERBOSE"))
        fprintf(stderr, "[wd] tuned stencil in=%d out=%d nrhs<=%d: R=%d threads=%d (%.3f ms/launch)\n", pin, pout,
                rhs_bucket(A.nrhs), *R, *th, best / 3);
    return WD_OK;
}

// WD_ETIMEOUT if a staged stencil launch gave up a bounded wait since the last check
int hop_err_check(wd_ctx *c) {
    int h = 0;
    WD_CUDA(cudaMemcpyAsync(&h, c->hop_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    WD_CUDA(cudaStreamSynchronize(c->st));
    if (h) {
        WD_CUDA(cudaMemsetAsync(c->hop_err, 0, sizeof(int), c->st));
        set_error("staged stencil: a bounded wait gave up");
        return WD_ETIMEOUT;
    }
    return WD_OK;
}

int hop(wd_ctx *c, int pin, int pout, int p, void *out, const void *in, const void *w, double a, double b,
        int nrhs, bool dag, const void *w2, double cc, const int *tsup, bool w2_ddl) {
    if (nrhs <= 0) return WD_OK;
    HopArgs A;
    A.out = out; A.in = in; A.w = w; A.w2 = w2; A.a = a; A.b = b; A.c = cc;
    A.err = c->hop_err;
    A.alist = c->alist; A.acount = c->acount;
    if (is_dd(pin)) {
        A.tsup = tsup;
        A.w2_ddl = w2_ddl ? 1 : 0;
    } else if (w2_ddl) {
        set_error("hop: a double-float addend needs the double-float stencil");
        return WD_EINVAL;
    }
    A.p = p; A.nrhs = nrhs; A.nrb = 1; A.g = c->g;
    // links in the precision of the input field; double-float: FP32 copy + remainder
    if (is_dd(pin)) {
        A.gauge = gauge_parity(c, P32, p);
        A.gauge_lo = (const char *)c->gauge_lo + (size_t)p * 8 * 9 * c->g.Vh * sizeof(float2);
    } else {
        A.gauge = gauge_parity(c, pin, p);
    }
    // algorithmic bytes: (in + out [+ w + w2]) spinors per RHS that does work
    // (inside a BiCGStab run: the RHS active at the last host check) + 8 links
    // per output site
    const double sb_in = spinor_bytes(pin), sb_out = spinor_bytes(pout);
    const int nwork = c->alist && c->act_count >= 0 && c->act_count < nrhs ? c->act_count : nrhs;
    const double bytes = (double)c->g.Vh *
                         (nwork * (sb_in + sb_out + (w ? sb_in : 0) + (w2 ? sb_in : 0)) + 8.0 * link_bytes(pin));
    int slot;
    prof_begin(c, pin == P64 || is_dd(pin) ? WD_K_HOP64 : WD_K_HOP, bytes, &slot);
    if (pin == PDD) {
        // FP64 input: split once into the double-float layout (part of this
        // stencil application's time; its bytes are not algorithmic)
        void *ddl;
        const int s = ws_get(c, "dd.in", field_bytes(c->g, P64, nrhs), &ddl);
        if (s != WD_OK) { prof_end(c, slot); return s; }
        cudaError_t e = launch_to_ddl(in, ddl, 12L * c->g.Vh * nrhs, c->st);
        c->launches++;
        if (e != cudaSuccess) { prof_end(c, slot); set_error("hop: %s", cudaGetErrorString(e)); return WD_ECUDA; }
        A.in = ddl;
    }
    int R, th;
    {
        const int s = tune_hop(c, pin, pout, A, dag, &R, &th);
        if (s != WD_OK) { prof_end(c, slot); return s; }
    }
    cudaError_t e = launch_hop_any(pin, pout, A, R, dag, th, c->st);
    if (e == cudaErrorNotSupported)   // an overridden variant that does not fit this shape
        e = launch_hop_any(pin, pout, A, c->hop_R[pin], dag, c->hop_threads[pin], c->st);
    prof_end(c, slot);
    c->launches++;
    if (e != cudaSuccess) { set_error("hop launch: %s", cudaGetErrorString(e)); return WD_ECUDA; }
    return WD_OK;
}

// ---- gauge ingest ---------------------------------------------------------
// From lexicographic FP64 links [4][V][3][3] to the eo doubled layout of one
// storage type: dir mu  = U_mu(x) (x bc[mu] if x_mu = L-1),
//               dir 4+mu = U_mu(x-mu)^dag (x bc[mu] if x_mu = 0).
template <typename G> struct LStore;
template <> struct LStore<double> {
    __device__ static void put(void *base, long idx, double re, double im) { ((double2 *)base)[idx] = make_double2(re, im); }
};
template <> struct LStore<float> {
    __device__ static void put(void *base, long idx, double re, double im) { ((float2 *)base)[idx] = make_float2((float)re, (float)im); }
};
template <> struct LStore<bf16> {
    __device__ static void put(void *base, long idx, double re, double im) {
        ((__nv_bfloat162 *)base)[idx] = __floats2bfloat162_rn((float)re, (float)im);
    }
};

// FP32 remainder of an FP64 link: U - (float)U, the low half of the
// double-float links (the high half is the FP32 copy)
struct LoTag {};
template <> struct LStore<LoTag> {
    __device__ static void put(void *base, long idx, double re, double im) {
        ((float2 *)base)[idx] = make_float2((float)(re - (double)(float)re), (float)(im - (double)(float)im));
    }
};

template <typename G>
__global__ void k_gauge_eo(const double *U, void *out, Geom g, int4 bc) {
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i >= (long)g.V) return;
    const int site = (int)i;
    int x = site % g.X, r = site / g.X;
    int y = r % g.Y; r /= g.Y;
    int z = r % g.Z, t = r / g.Z;
    const int p = (x + y + z + t) & 1, s = site >> 1;
    const int c[4] = {x, y, z, t};
    const int L[4] = {g.X, g.Y, g.Z, g.T};
    const int b[4] = {bc.x, bc.y, bc.z, bc.w};
    const long Vh = g.Vh;
    void *base = (char *)out;
    for (int mu = 0; mu < 4; ++mu) {
        // forward link U_mu(x)
        const double *u = U + ((size_t)mu * g.V + site) * 18;
        const double sf = (c[mu] == L[mu] - 1) ? b[mu] : 1;
        const long dbase = ((long)p * 8 + mu) * 9 * Vh;
        for (int k = 0; k < 9; ++k) LStore<G>::put(base, dbase + k * Vh + s, sf * u[2 * k], sf * u[2 * k + 1]);
        // backward link U_mu(x-mu)^dag
        int cm[4] = {x, y, z, t};
        cm[mu] = c[mu] == 0 ? L[mu] - 1 : c[mu] - 1;
        const int sm = cm[0] + g.X * (cm[1] + g.Y * (cm[2] + g.Z * cm[3]));
        const double *um = U + ((size_t)mu * g.V + sm) * 18;
        const double sb = (c[mu] == 0) ? b[mu] : 1;
        const long bbase = ((long)p * 8 + 4 + mu) * 9 * Vh;
        for (int a = 0; a < 3; ++a)
            for (int bb = 0; bb < 3; ++bb) {
                // (U^dag)_{a b} = conj(U_{b a})
                const int k = 3 * bb + a;
                LStore<G>::put(base, bbase + (3 * a + bb) * Vh + s, sb * um[2 * k], -sb * um[2 * k + 1]);
            }
    }
}

static int ingest_gauge(wd_ctx *c, const double *gauge_host) {
    const size_t n = (size_t)4 * c->g.V * 18;
    double *dU;
    WD_TRY(ws_get(c, "gauge.lex", n * sizeof(double), (void **)&dU));
    WD_CUDA(cudaMemcpyAsync(dU, gauge_host, n * sizeof(double), cudaMemcpyDefault, c->st));
    const int4 bc = make_int4(c->bc[0], c->bc[1], c->bc[2], c->bc[3]);
    const unsigned blocks = (unsigned)((c->g.V + 127) / 128);
    k_gauge_eo<double><<<blocks, 128, 0, c->st>>>(dU, c->gauge[P64], c->g, bc);
    k_gauge_eo<float><<<blocks, 128, 0, c->st>>>(dU, c->gauge[P32], c->g, bc);
    k_gauge_eo<bf16><<<blocks, 128, 0, c->st>>>(dU, c->gauge[P16], c->g, bc);
    k_gauge_eo<LoTag><<<blocks, 128, 0, c->st>>>(dU, c->gauge_lo, c->g, bc);
    c->launches += 4;
    WD_CUDA(cudaGetLastError());
    WD_CUDA(cudaStreamSynchronize(c->st));
    return WD_OK;
}

}  // namespace wd

using namespace wd;

extern "C" const char *wd_last_error(void) { return wd::g_err; }

extern "C" int wd_create(wd_ctx **out, const int dims[4], const double *gauge, double kappa, const int bc[4],
                         void *stream) {
    if (!out || !dims || !gauge || !bc) { set_error("wd_create: null argument"); return WD_EINVAL; }
    *out = nullptr;
    long V = 1;
    for (int m = 0; m < 4; ++m) {
        if (dims[m] < 2 || dims[m] % 2) { set_error("wd_create: extent %d of direction %d must be even and >= 2", dims[m], m); return WD_EINVAL; }
        if (bc[m] != 1 && bc[m] != -1) { set_error("wd_create: bc[%d] must be +1 or -1", m); return WD_EINVAL; }
        V *= dims[m];
    }
    if (V > (1L << 30)) { set_error("wd_create: lattice too large"); return WD_EINVAL; }
    wd_ctx *c = new wd_ctx();
    for (int m = 0; m < 4; ++m) { c->dims[m] = dims[m]; c->bc[m] = bc[m]; }
    c->kappa = kappa;
    c->g.X = dims[0]; c->g.Y = dims[1]; c->g.Z = dims[2]; c->g.T = dims[3];
    c->g.Xh = dims[0] / 2; c->g.V = (int)V; c->g.Vh = (int)(V / 2);
    c->st = (cudaStream_t)stream;
    c->launches = 0;
    c->prof = false;
    c->mg = nullptr;
    c->mg3 = nullptr;
    c->last_n2 = 0;
    for (int p = 0; p < 5; ++p) { c->hop_R[p] = p == P64 || is_dd(p) ? 1 : 2; c->hop_threads[p] = 128; }
    for (int p = 0; p < 3; ++p) c->gauge[p] = nullptr;
    c->gauge_lo = nullptr;
    {
        const char *e = getenv("WD_DD");
        c->outer = e && atoi(e) == 0 ? P64 : PDD;
    }
    c->autotune = getenv("WD_NO_AUTOTUNE") == nullptr;
    c->hop_err = nullptr;
    c->alist = nullptr;
    c->acount = nullptr;
    c->gst = nullptr;
    c->loop_dev = nullptr;
    c->graph_off = false;
    c->act_count = -1;
    c->noalloc_scratch = nullptr;
    if (cudaMalloc(&c->hop_err, sizeof(int)) != cudaSuccess || cudaMemset(c->hop_err, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        set_error("wd_create: allocation failed");
        wd_destroy(c);
        return WD_ENOMEM;
    }
    const size_t nl = (size_t)2 * 8 * 9 * c->g.Vh;
    const size_t eb[3] = {16, 8, 4};
    for (int p = 0; p < 3; ++p) {
        if (cudaMalloc(&c->gauge[p], nl * eb[p]) != cudaSuccess) {
            cudaGetLastError();
            set_error("wd_create: link allocation failed");
            wd_destroy(c);
            return WD_ENOMEM;
        }
    }
    if (cudaMalloc(&c->gauge_lo, nl * 8) != cudaSuccess) {
        cudaGetLastError();
        set_error("wd_create: link allocation failed");
        wd_destroy(c);
        return WD_ENOMEM;
    }
    int s = ingest_gauge(c, gauge);
    if (s != WD_OK) { wd_destroy(c); return s; }
    // resolve the static array of wd_apply_noalloc here, with the context's
    // device current: this loads its module (which holds the array) now, so
    // that the allocation-free calls later find it in place
    s = noalloc_scratch_ptr(&c->noalloc_scratch);
    if (s != WD_OK) { wd_destroy(c); return s; }
    *out = c;
    return WD_OK;
}

extern "C" int wd_update_gauge(wd_ctx *c, const double *gauge, double kappa) {
    if (!c || !gauge) { set_error("wd_update_gauge: null argument"); return WD_EINVAL; }
    c->kappa = kappa;
    return ingest_gauge(c, gauge);
}

void wd_mg_free(wd_ctx *c);
namespace wd { void wd_loops_free(wd_ctx *c); }

extern "C" int wd_destroy(wd_ctx *c) {
    if (!c) return WD_OK;
    cudaStreamSynchronize(c->st);
    wd_mg_free(c);
    wd_loops_free(c);
    for (int p = 0; p < 3; ++p) if (c->gauge[p]) cudaFree(c->gauge[p]);
    if (c->gauge_lo) cudaFree(c->gauge_lo);
    if (c->hop_err) cudaFree(c->hop_err);
    for (auto &b : c->bufs) cudaFree(b.second.first);
    for (auto &b : c->hbufs) cudaFreeHost(b.second.first);
    for (auto &r : c->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    delete c;
    return WD_OK;
}

extern "C" int wd_apply(wd_ctx *c, const void *in, void *out, int nrhs, int prec, int dagger) {
    if (!c || (!in && nrhs > 0) || (!out && nrhs > 0) || nrhs < 0) { set_error("wd_apply: bad argument"); return WD_EINVAL; }
    if (prec < 0 || prec > 3) { set_error("wd_apply: bad precision %d", prec); return WD_EINVAL; }
    if (nrhs == 0) return WD_OK;
    const int pf = prec;               // field storage inside the stencil (PDD: FP64 fields)
    const int po = prec == P64 || prec == PDD ? prec : P32;
    const bool udbl = prec == P64 || prec == PDD;
    const size_t fin = field_bytes(c->g, pf, nrhs), fout = field_bytes(c->g, po, nrhs);
    void *ie, *io, *oe, *oo;
    WD_TRY(ws_get(c, "apply.ie", fin, &ie));
    WD_TRY(ws_get(c, "apply.io", fin, &io));
    WD_TRY(ws_get(c, "apply.oe", fout, &oe));
    WD_TRY(ws_get(c, "apply.oo", fout, &oo));
    WD_TRY(user_to_eo(c, in, udbl, pf == PDD ? P64 : pf, ie, io, nrhs));
    // (D x)_e = x_e - k H_eo x_o,  (D x)_o = x_o - k H_oe x_e
    const double k = c->kappa;
    WD_TRY(hop(c, pf, po, 0, oe, io, ie, 1.0, -k, nrhs, dagger != 0));
    WD_TRY(hop(c, pf, po, 1, oo, ie, io, 1.0, -k, nrhs, dagger != 0));
    WD_TRY(eo_to_user(c, oe, oo, po == PDD ? P64 : po, out, udbl, nrhs));
    WD_CUDA(cudaGetLastError());
    return WD_OK;
}

extern "C" int wd_solve(wd_ctx *c, const double *rhs, double *x, int nrhs, double tol, int prec, int max_iter,
                        int *iters_out, double *true_resid_out) {
    if (!c || nrhs < 0 || ((!rhs || !x) && nrhs > 0) || !(tol > 0) || max_iter < 1 || prec < 0 || prec > 2) {
        set_error("wd_solve: bad argument");
        return WD_EINVAL;
    }
    if (nrhs == 0) return WD_OK;
    const size_t f = field_bytes(c->g, P64, nrhs);
    double *be, *bo, *xe, *xo;
    WD_TRY(ws_get(c, "solve.be", f, (void **)&be));
    WD_TRY(ws_get(c, "solve.bo", f, (void **)&bo));
    WD_TRY(ws_get(c, "solve.xe", f, (void **)&xe));
    WD_TRY(ws_get(c, "solve.xo", f, (void **)&xo));
    WD_TRY(user_to_eo(c, rhs, true, P64, be, bo, nrhs));
    int s = solve_eo(c, be, bo, xe, xo, nrhs, tol, prec, max_iter, iters_out, true_resid_out);
    if (s != WD_OK && s != WD_ENOCONV && s != WD_EBREAKDOWN) return s;
    WD_TRY(eo_to_user(c, xe, xo, P64, x, true, nrhs));
    WD_CUDA(cudaStreamSynchronize(c->st));
    return s;
}

extern "C" int wd_profile(wd_ctx *c, int enable) {
    if (!c) return WD_EINVAL;
    WD_CUDA(cudaStreamSynchronize(c->st));
    if (enable) {
        for (auto &r : c->recs) { c->event_pool.push_back(r.a); c->event_pool.push_back(r.b); }
        c->recs.clear();
    }
    c->prof = enable != 0;
    return WD_OK;
}

extern "C" int wd_profile_get(wd_ctx *c, int kernel, int64_t *launches, double *ms, double *bytes) {
    if (!c || kernel < 0 || kernel >= WD_K_COUNT) return WD_EINVAL;
    WD_CUDA(cudaStreamSynchronize(c->st));
    int64_t n = 0;
    double t = 0, b = 0;
    for (auto &r : c->recs) {
        if (r.kernel != kernel) continue;
        float e = 0;
        if (cudaEventElapsedTime(&e, r.a, r.b) == cudaSuccess) { t += e; b += r.bytes; ++n; }
        else cudaGetLastError();
    }
    if (launches) *launches = n;
    if (ms) *ms = t;
    if (bytes) *bytes = b;
    return WD_OK;
}

extern "C" int64_t wd_launch_count(wd_ctx *c) { return c ? c->launches : 0; }
