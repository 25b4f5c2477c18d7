// Internal declarations of libwd (not part of the C ABI).
#pragma once
#include <map>
#include <string>
#include <vector>

#include "../../include/wd.h"
#include "wd_common.cuh"

namespace wd {

// ---- errors ----------------------------------------------------------------
void set_error(const char *fmt, ...);
#define WD_CUDA(expr)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            ::wd::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(e_)); \
            return WD_ECUDA;                                                               \
        }                                                                                  \
    } while (0)
#define WD_TRY(expr)                 \
    do {                             \
        int s_ = (expr);             \
        if (s_ != WD_OK) return s_;  \
    } while (0)

// ---- kernels ---------------------------------------------------------------
struct HopArgs {
    void *out;             // output parity field (rhs 0)
    const void *in;        // input field of the other parity
    const void *w;         // same-parity addend (nullable)
    const void *w2;        // second same-parity addend (nullable)
    const void *gauge;     // links of the output parity: [8][9][Vh]
    const void *gauge_lo = nullptr;   // FP32 remainders of the FP64 links (double-float stencil)
    double a, b, c;        // out = a*w + c*w2 + b*H(in)
    int p;                 // output parity
    int nrhs, nrb;
    Geom g;
    int *err = nullptr;    // error flag of the staged variant (bounded waits); set by hop()
    // Inside a BiCGStab run: the RHS still working, ascending (alist[0 ..
    // *acount)); RHS tiles walk this list, so converged RHS cost nothing.
    // Null: all nrhs RHS.
    const int *alist = nullptr;
    const int *acount = nullptr;
    // timeslice that holds the whole input of each RHS (nullable; entry -1:
    // anywhere): output sites more than one timeslice away get no hop term
    // (double-float stencil only; time-diluted and point sources)
    const int *tsup = nullptr;
    // double-float stencil only: the second addend w2 is a double-float
    // layout field (float4 (re.h, im.h, re.l, im.l) per complex) instead of FP64
    int w2_ddl = 0;
    // block order of the FP32/BF16 stencil: 0 = RHS tile fastest (the site
    // tiles of all RHS run together), 1 = site tile fastest (the resident
    // blocks sweep a few whole RHS fields at a time)
    int rhs_major = 0;
};

// true if the hop can reach output timeslice t from RHS rhs's input support
__device__ __forceinline__ bool hop_reaches(const HopArgs &A, int rhs, int t) {
    if (A.tsup == nullptr) return true;
    const int t0 = __ldg(A.tsup + rhs);
    if (t0 < 0) return true;
    const int dt = t > t0 ? t - t0 : t0 - t;
    return dt <= 1 || dt == A.g.T - 1;
}

// Programmatic dependent launch: a kernel launched with launch_pdl may be
// scheduled while its predecessor on the stream is still finishing; it must
// call pdl_wait() before touching any memory, which returns once the
// predecessor has completed and its writes are visible (a no-op for a normal
// launch).  Hides the launch gap between the dependent kernels of a Krylov
// iteration.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// RHS handled by slot r of RHS tile rb (R slots per tile), or -1 if none
__device__ __forceinline__ int tile_rhs(const HopArgs &A, int rb, int r, int R) {
    const int k = rb * R + r;
    if (A.alist == nullptr) return k < A.nrhs ? k : -1;
    return k < __ldg(A.acount) ? __ldg(A.alist + k) : -1;
}

template <typename SIn, typename SOut, typename SW, typename G>
cudaError_t launch_hop(const HopArgs &A, int R, bool dag, int threads, cudaStream_t st);

// Double-float stencil (wd_dslash_dd.cu): A.in in the double-float layout
// (FP64 eo layout, each complex as float4 (re.h, im.h, re.l, im.l)), addends
// FP64, output FP64 or (out_dd) double-float layout.  R = 1, 2 scalar; 11, 12
// packed f32x2.
cudaError_t launch_hop_dd(const HopArgs &A, int R, bool dag, int threads, bool out_dd, cudaStream_t st);
// FP64 eo field -> double-float layout, n complex numbers
cudaError_t launch_to_ddl(const void *in, void *out, long n, cudaStream_t st);

// several lattices' stencils in one persistent launch (FP32 arithmetic only)
static constexpr int WD_MAX_BATCH = 8;
struct HopBatch {
    HopArgs job[WD_MAX_BATCH];
    int blocks[WD_MAX_BATCH];
    int njobs, total;
};
template <typename SIn, typename SOut, typename SW, typename G>
cudaError_t launch_hop_batched(HopBatch B, int R, cudaStream_t st);

// Precision tags of the inner solve.  Stencil-only tags for the FP64 steps of
// the mixed-precision solves (double-float arithmetic): PDD = FP64 storage,
// PDDL = double-float layout (same bytes per site).
enum Prec { P64 = 0, P32 = 1, P16 = 2, PDD = 3, PDDL = 4 };
inline bool is_dd(int prec) { return prec == PDD || prec == PDDL; }

// Bytes of one site-spinor (12 complex) and one link (9 complex) per storage
inline int spinor_bytes(int prec) { return prec == P64 || is_dd(prec) ? 192 : prec == P32 ? 96 : 48; }
inline int link_bytes(int prec) { return prec == P64 || is_dd(prec) ? 144 : prec == P32 ? 72 : 36; }

// BiCGStab per-RHS state, FP64 scalars
struct BiState {
    double2 rho, alpha, omega, beta;
    double rr, bb, thr;    // |r|^2, |b|^2, convergence threshold on |r|^2
    int active, flag, iters, pad;
};
static_assert(sizeof(BiState) % sizeof(int) == 0, "the activity mask strides BiState in ints");

}  // namespace wd

// ---- context ---------------------------------------------------------------
struct wd_prof_rec {
    cudaEvent_t a, b;
    int kernel;
    double bytes;
};

// A BiCGStab loop captured as a CUDA graph (wd_solver.cu): a conditional
// while node around two iterations, keyed by everything its kernels see
struct wd_loop_graph {
    std::vector<uintptr_t> key;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int kernels;                    // kernel launches per body (two iterations + condition)
};

// third multigrid level (wd_mg3.cu): level-2 sites aggregated by agg2
struct wd_mg3 {
    int nv2, ncd2;
    int agg2[4], cd3[4];
    int Vcc;
    double2 *P2;       // [Vc][ncd][nv2]: column k of the half of coarse dof i
    double2 *D3;       // [Vcc][9][ncd2][ncd2]
    int *nbr3;         // [Vcc][9]
};

// Probing on the coarse level (wd_mlmc.cu): colour (sigma . X) mod nc of the
// coarse site X (coarse extents cd), times dilution over the dil coarse dofs
// of a site (dil = 1: none); m = nc * dil vectors per noise sample
struct CoarseProbe {
    int nc, sigma[4], cd[4], dil, m;
};

// multigrid state (wd_mg.cu)
struct wd_mg {
    int nv, ncd;
    int agg[4], cd[4];
    int Vc;
    double2 *P;        // [2][Vh][12][nv]
    double2 *Dc;       // [Vc][9][ncd][ncd]
    int *nbr;          // [Vc][9]
    void *Wtc;         // tensor-core block operand (bf16): [Vc][9 ncd/16][ncd][32], built by wd_coarse_tc.cu
    void *Wlo;         // its rounding remainder (bf16): Wtc + Wlo carries ~16 significant bits
    int tc_sms;        // SMs of the device (one persistent tensor-core CTA each)
    float2 *Dc32;      // [Vc][9][ncd][ncd] complex64 copy for the FP32 CUDA-core path
    float2 *Dclo;      // Dc - Dc32 as complex64: with Dc32 the double-float blocks of the FP64 residual
    float2 *Phi, *Plo; // P as double-float pairs (FP32 copy and remainder), for the prolongation
    double2 *Gt;       // [Vc][agg_t][2][nv][nv]: Gram matrices of P's columns restricted to one
                       // timeslice of an aggregate and one chirality half (coarse contractions)
    float2 *Ghi, *Glo; // Gt as double-float pairs
};

struct wd_ctx {
    int dims[4];
    int bc[4];
    double kappa;
    wd::Geom g;
    cudaStream_t st;
    void *gauge[3];                 // eo doubled links per precision P64/P32/P16: [2][8][9][Vh]
    void *gauge_lo;                 // FP64 link minus its FP32 copy, as FP32: [2][8][9][Vh] float2
    int outer;                      // stencil of the FP64 steps of mixed solves: PDD, or P64 (WD_DD=0)
    std::map<std::string, std::pair<void *, size_t>> bufs;   // named device workspaces
    std::map<std::string, std::pair<void *, size_t>> hbufs;  // named pinned host workspaces
    int64_t launches;
    bool prof;
    std::vector<wd_prof_rec> recs;
    std::vector<cudaEvent_t> event_pool;
    int hop_R[5];                   // default RHS tile per input precision
    int hop_threads[5];
    bool autotune;                  // time the stencil launch shapes on first use
    int *hop_err;                   // device flag: a staged stencil wait gave up
    const int *alist;               // active-RHS list of the running BiCGStab (nullable)
    const int *acount;              // its length (device)
    int act_count;                  // RHS active at the last host check (-1: unknown), for profiled bytes
    std::vector<wd_loop_graph> loops;   // captured BiCGStab loops (most recent last)
    cudaStream_t gst;               // capture stream of those graphs
    int *loop_dev;                  // [iterations run, iteration limit] of a graph launch
    bool graph_off;                 // a graph call failed: plain loops from then on
    std::map<int, std::pair<int, int>> tuned;   // (pin, pout, RHS bucket) -> (R, threads)
    void *noalloc_scratch;          // device address of the static array of wd_apply_noalloc on this
                                    // context's device (resolved by wd_create)
    wd_mg *mg;
    wd_mg3 *mg3;                    // third level (built on mg), nullable
    std::vector<double> last_level2;    // [n2][T][2]
    int last_n2;
};

namespace wd {
// device workspace by name, grown on demand (contents undefined after growth)
int ws_get(wd_ctx *c, const char *name, size_t bytes, void **out);
int hws_get(wd_ctx *c, const char *name, size_t bytes, void **out);
// profiling brackets around one launch of kernel family `k` moving `bytes`
void prof_begin(wd_ctx *c, int k, double bytes, int *slot);
void prof_end(wd_ctx *c, int slot);

// Launch one hop on the context's links: out(parity p) = a*w + c*w2 + b*H(in)
// for inner precision prec; SIn is the input storage, SOut the output storage.
int hop(wd_ctx *c, int prec_in, int prec_out, int p, void *out, const void *in, const void *w,
        double a, double b, int nrhs, bool dag = false, const void *w2 = nullptr, double cc = 0.0,
        const int *tsup = nullptr, bool w2_ddl = false);

int hop_err_check(wd_ctx *c);

// Device address of the static staging array of wd_apply_noalloc on the
// current device (wd_noalloc.cu); called by wd_create, which is where that
// array's module is loaded and the array comes into being.
int noalloc_scratch_ptr(void **out);

// layout conversions between the user layout and the eo layout
int user_to_eo(wd_ctx *c, const void *user, bool user_double, int prec, void *even, void *odd, int nrhs);
int eo_to_user(wd_ctx *c, const void *even, const void *odd, int prec, void *user, bool user_double, int nrhs);

// Solver core on eo fields (wd_solver.cu).  b: FP64 eo [2 parities] fields.
// src_tsup (device [nrhs], nullable): timeslice holding each RHS's source
// (-1: anywhere).  x_odd nullable: no odd-site reconstruction (then
// resid_out must be null); bhat_out: the Schur source b_e + k H_eo b_o
// (a workspace of the context, valid until the next solve).
// the same entirely in FP32 for tol >= 1e-6 (no FP64 certification)
int solve_eo_fp32(wd_ctx *c, const double *b_e, const double *b_o, double *x_e, double *x_o, int nrhs, double tol);
int solve_eo(wd_ctx *c, const double *b_even, const double *b_odd, double *x_even, double *x_odd, int nrhs,
             double tol, int prec, int max_iter, int *iters_out, double *resid_out, const int *src_tsup = nullptr,
             const double **bhat_out = nullptr);

// blas (wd_blas.cu)
// A vector space for BLAS-1: `units` 12-complex units per right-hand side, in
// the eo chunk layout (flat = false, units = Vh) or the plain layout
// [rhs][unit][12] (flat = true, coarse-grid vectors).
struct Space {
    long units;
    bool flat;
};
inline Space fine_space(const Geom &g) { Space s; s.units = g.Vh; s.flat = false; return s; }
inline size_t space_bytes(const Space &s, int prec, int nrhs) { return (size_t)nrhs * s.units * spinor_bytes(prec); }
size_t field_bytes(const Geom &g, int prec, int nrhs);   // one parity of a fine field
int blas_copy_convert(wd_ctx *c, const Space &sp, int prec_src, const void *src, int prec_dst, void *dst, int nrhs,
                      const double *scale_dev);
// x (double-float layout) += scale[rhs] * e (FP32), in double-float arithmetic
int blas_axpy_ddl(wd_ctx *c, const Space &sp, void *x_ddl, const void *e32, const double *scale_dev, int nrhs);
// FP64 copy of a double-float layout field (integer assembly, within one FP64 ulp)
int blas_ddl_to_f64(wd_ctx *c, const Space &sp, const void *x_ddl, double *x64, int nrhs);
int blas_axpy_mixed(wd_ctx *c, const Space &sp, double *x64, int prec_e, const void *e, const double *scale_dev,
                    int nrhs);
int blas_norm2(wd_ctx *c, const Space &sp, int prec, const void *a, int nrhs, double *out_dev);
int blas_zero(wd_ctx *c, void *p, size_t bytes);

// out = A in for one operator, in the precisions the solver set up
typedef int (*OpFn)(wd_ctx *c, const void *in, void *out, int nrhs, void *user);
// r = b - A x in FP64
typedef int (*ResFn)(wd_ctx *c, const double *b, const double *x, double *r, int nrhs, void *user);

// BiCGStab building blocks (wd_blas.cu)
struct BiVecs {
    void *x, *r, *rh, *v, *t;   // working precision (SW)
    void *p, *s;                // operator-input precision (SP)
    BiState *st;
    double *part;               // reduction partials
    int *count;                 // active count (device)
    int *alist;                 // active RHS, ascending (device, count entries)
    int bpr;                    // reduction blocks per RHS
    Space sp;
    OpFn op;
    void *op_user;
    // the operator's launches may be captured in a graph; sig: what of
    // op_user its kernels see (precisions, workspace), part of the graph key
    bool graph_ok = false;
    uintptr_t sig[3] = {0, 0, 0};
};
int bicg_init(wd_ctx *c, int pw, int pp, BiVecs &V, const void *b, int nrhs, double tol_rel,
              const double *bnorm2_dev);
int bicg_iter(wd_ctx *c, int pw, int pp, BiVecs &V, int nrhs);
int bicg_after_v(wd_ctx *c, int pw, int pp, BiVecs &V, int nrhs);
int bicg_after_t(wd_ctx *c, int pw, int pp, BiVecs &V, int nrhs);
int reduction_bpr(long units, int nrhs);
int alloc_bivecs(wd_ctx *c, const Space &sp, int pw, int pp, int nrhs, BiVecs &V, const std::string &tag);

// Defect-correction (or plain FP64) BiCGStab solve of A x = b on one space
// (wd_solver.cu).  b, x: FP64 vectors of the space (x overwritten).
struct Problem {
    Space sp;
    OpFn op64;  void *u64;      // FP64 operator (FP64 mode)
    OpFn oplo;  void *ulo;      // inner operator, inputs in pp, outputs in pw
    ResFn res64; void *ures;    // FP64 residual
    // res64 writes the residual in the double-float layout (PDDL) instead of
    // FP64: its norm and its FP32 copy then run on the FP32 pipes
    bool res_ddl = false;
    // the solution is kept in the double-float layout during the outer loop
    // (res64 then reads x in that layout; FP64 x is written once at the end)
    bool x_ddl = false;
    const char *tag;            // workspace name prefix
    bool graph_ok = false;      // operators capturable in a graph (sig64 / siglo: their keys)
    uintptr_t sig64[3] = {0, 0, 0}, siglo[3] = {0, 0, 0};
    double inner_tol = 0.0;     // tolerance of the inner solves (0: by inner precision)
    // Recursive residual update r <- r - |r| opupd(e), e the inner solution of
    // the normalised residual (inner precision in and out, FP64 sum), in place
    // of res64 once the residual is small: the update adds at most
    // upd_err |r| to r (upd_err: a bound on the normwise error of opupd
    // relative to |r|), so it is taken while upd_err |r| <= tol |b| / 4, and
    // each RHS counts as converged only when its residual plus the sum of
    // these bounds is <= tol |b|.  The residual may be FP64 or the
    // double-float layout (res_ddl).
    OpFn opupd = nullptr; void *uupd = nullptr;
    double upd_err = 0.0;
};
// restriction P^dag v and prolongation P y between eo FP64 fine fields and
// coarse FP64 vectors (wd_mg.cu); dd_ok: double-float arithmetic allowed
// (~2^-44 relative, for the estimators), else FP64
int mg_restrict_eo(wd_ctx *c, const double *ve, const double *vo, double *yc, int nrhs, bool dd_ok = false);
int mg_prolong_eo(wd_ctx *c, const double *yc, double *ve, double *vo, int nrhs, bool dd_ok = false);
// per-timeslice contraction of coarse vectors: part[r][t] = sum_{x in t}
// (P a_r)(x)^dag B (P b_r)(x), B = 1 or g5, evaluated on the coarse lattice
// from the Gram matrices Gt (wd_mg.cu); part: device complex [nrhs][T]
int mg_contract_coarse_t(wd_ctx *c, const double *a, const double *b, int gamma5, int nrhs, double *part);
// per-timeslice restriction Rt[r][X][tau][i] (complex FP64, tau the timeslice
// inside aggregate X) of eo FP64 fields, and yc = sum_tau Rt = P^dag v
int mg_restrict_t_eo(wd_ctx *c, const double *ve, const double *vo, double *Rt, double *yc, int nrhs);
// the same for the plain Rademacher noise of samples sample0 .. sample0 +
// nrhs - 1 of seed (the fields gen_noise_eo writes, passed as ve, vo for the
// FP64 path): in double-float arithmetic from the noise's sign words
int mg_restrict_t_noise(wd_ctx *c, uint64_t seed, int sample0, const double *ve, const double *vo, double *Rt,
                        double *yc, int nrhs);
// part[r][t] = sum_{x in t} v_r(x)^dag B (P y_r)(x) from the per-timeslice
// restriction Rt of v (B = 1 or g5); part: device complex [nrhs][T]
int mg_contract_rt(wd_ctx *c, const double *Rt, const double *y, int gamma5, int nrhs, double *part);
int dc_solve(wd_ctx *c, const Problem &P, const double *b, double *x, int nrhs, const double *bnorm2_dev,
             const std::vector<double> &bnorm2, double tol, int prec, int max_iter, std::vector<int> &iters,
             std::vector<double> &last_rn2);
}  // namespace wd
