// wd_apply_noalloc: D x (or D^dag x) like wd_apply, without allocating.
//
// Some callers cannot allocate device memory once they are running: services
// that reserve their whole device-memory budget at start-up (a later
// cudaMalloc fails or is forbidden by policy), and frameworks whose caching
// allocator must own every byte of device memory (an allocation behind its
// back can exhaust or fragment the pool it manages).  wd_apply stages the
// fields in even-odd order in buffers the context allocates on first use;
// this variant stages them in one file-scope device array instead, so a call
// allocates nothing.
//
// The array holds WD_NOALLOC_SCRATCH_BYTES (64 MiB) on every GPU on which a
// context is created, until the process exits.  With lazy module loading the
// CUDA runtime creates a module's device arrays when the module is first
// used, so wd_create resolves the array's device address (once per device,
// with the context's device current) and keeps it in the context: the array
// exists from wd_create on, and the entry point itself allocates nothing and
// stages on the context's own device whichever device is current.  Every
// call uses the same array and leaves its contents behind; the staging fields
// are fully overwritten before they are read, so nothing needs clearing, but
// two calls whose work overlaps on the GPU (different streams, or different
// host threads) race on the array.
#include <mutex>

#include "wd_internal.h"

#define WD_NOALLOC_SCRATCH_BYTES (64u << 20)
#define WD_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char wd_noalloc_scratch[WD_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_mu;
void *g_scratch[WD_NOALLOC_MAX_DEVICES];
}  // namespace

using namespace wd;

namespace wd {
int noalloc_scratch_ptr(void **out) {
    int dev = 0;
    WD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= WD_NOALLOC_MAX_DEVICES) {
        set_error("wd_apply_noalloc: device ordinal %d beyond %d", dev, WD_NOALLOC_MAX_DEVICES);
        return WD_ENOTSUP;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, wd_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error("wd_apply_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return WD_ECUDA;
        }
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    return WD_OK;
}
}  // namespace wd

extern "C" int wd_apply_noalloc(wd_ctx *c, const void *in, void *out, int nrhs, int prec, int dagger) {
    if (!c || nrhs < 0 || ((!in || !out) && nrhs > 0) || prec < 0 || prec > 2) {
        set_error("wd_apply_noalloc: bad argument");
        return WD_EINVAL;
    }
    if (nrhs == 0) return WD_OK;
    const int pf = prec, po = prec == P64 ? P64 : P32;
    const size_t fin = field_bytes(c->g, pf, nrhs), fout = field_bytes(c->g, po, nrhs);
    // four staging fields, each rounded up to 256 bytes
    const size_t a_in = (fin + 255) & ~(size_t)255, a_out = (fout + 255) & ~(size_t)255;
    const size_t need = 2 * a_in + 2 * a_out;
    if (need > WD_NOALLOC_SCRATCH_BYTES) {
        set_error("wd_apply_noalloc: %d right-hand sides on this lattice need %zu bytes of staging, "
                  "more than the %u-byte static scratch; use wd_apply or fewer right-hand sides",
                  nrhs, need, WD_NOALLOC_SCRATCH_BYTES);
        return WD_EINVAL;
    }
    unsigned char *base = (unsigned char *)c->noalloc_scratch;
    if (!base) {
        set_error("wd_apply_noalloc: the context has no static staging array");
        return WD_ENOTSUP;
    }
    void *ie = base, *io = base + a_in, *oe = base + 2 * a_in, *oo = base + 2 * a_in + a_out;
    const bool udbl = prec == P64;
    WD_TRY(user_to_eo(c, in, udbl, pf, ie, io, nrhs));
    const size_t per = (size_t)8 * 9 * c->g.Vh * (pf == P64 ? 16 : pf == P32 ? 8 : 4);
    HopArgs A;
    A.a = 1.0; A.b = -c->kappa; A.c = 0.0; A.w2 = nullptr; A.nrhs = nrhs; A.nrb = 1; A.g = c->g;
    A.err = c->hop_err;
    const int R = c->hop_R[pf], th = c->hop_threads[pf];
    for (int p = 0; p < 2; ++p) {
        // (D x)_p = x_p - kappa H_{p,1-p} x_{1-p}
        A.p = p;
        A.out = p ? oo : oe;
        A.in = p ? ie : io;
        A.w = p ? io : ie;
        A.gauge = (const char *)c->gauge[pf] + p * per;
        cudaError_t e;
        if (pf == P64) e = launch_hop<double, double, double, double>(A, R, dagger != 0, th, c->st);
        else if (pf == P32) e = launch_hop<float, float, float, float>(A, R, dagger != 0, th, c->st);
        else e = launch_hop<bf16, float, bf16, bf16>(A, R, dagger != 0, th, c->st);
        c->launches++;
        if (e != cudaSuccess) { set_error("wd_apply_noalloc: %s", cudaGetErrorString(e)); return WD_ECUDA; }
    }
    WD_TRY(eo_to_user(c, oe, oo, po, out, udbl, nrhs));
    return WD_OK;
}
