// Internal declarations of the CCGF library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>
#include "../../include/ccgf.h"

typedef long long i64;

// ----------------------------------------------------------------------------- errors
void set_last_error(const std::string &msg);
#define CCGF_CUDA_TRY(expr)                                                                    \
    do {                                                                                       \
        cudaError_t _e = (expr);                                                               \
        if (_e != cudaSuccess) {                                                               \
            set_last_error(std::string(#expr) + ": " + cudaGetErrorString(_e));                \
            return _e == cudaErrorMemoryAllocation ? CCGF_ERR_OOM : CCGF_ERR_CUDA;             \
        }                                                                                      \
    } while (0)
#define CCGF_TRY(expr)                                                                         \
    do {                                                                                       \
        ccgf_status _s = (expr);                                                               \
        if (_s != CCGF_OK) return _s;                                                          \
    } while (0)

// ----------------------------------------------------------------------------- complex types
template <typename R> struct cvec;
template <> struct cvec<double> { typedef double2 T; };
template <> struct cvec<float> { typedef float2 T; };

// ----------------------------------------------------------------------------- device buffers
// Owning device buffer: freed by its destructor, so every early return of a function frees the
// buffers it allocated; movable, not copyable.
template <typename T> struct DBuf {
    T *p = nullptr;
    i64 n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n) {
        o.p = nullptr;
        o.n = 0;
    }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            n = o.n;
            o.p = nullptr;
            o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};
ccgf_status dalloc_bytes(void **p, size_t bytes);
template <typename T> ccgf_status dalloc(DBuf<T> &b, i64 n) {
    b.release();
    ccgf_status s = dalloc_bytes((void **)&b.p, (size_t)(n > 0 ? n : 1) * sizeof(T));
    b.n = s == CCGF_OK ? n : 0;
    return s;
}
template <typename T> void dfree(DBuf<T> &b) { b.release(); }

// Runs a cleanup on every exit path of a scope (pinned host memory, events).
template <typename F> struct ScopeExit {
    F f;
    ~ScopeExit() { f(); }
};
template <typename F> ScopeExit<F> on_scope_exit(F f) { return ScopeExit<F>{f}; }

// ----------------------------------------------------------------------------- batched GEMM
// C_b = alpha * sum_{r<nred} A_{b,r} B_{b,r} + beta * C_b,  complex, b < batch.
// A_{b,r}[m,k] = A0[offA[b*nred+r] + m*rsA + k*csA], likewise B[k,n], C[m,n].
struct GemmDesc {
    int M, N, K, nred, batch;
    i64 rsA, csA, rsB, csB, rsC, csC;
    const i64 *offA, *offB, *offC;   // device offset tables
    double2 alpha, beta;
    int tile;                        // SIMT per-thread tile: 0 = the launcher's model choice, k = its k-th candidate
    int ksplit;                      // SIMT split of K across CTAs: 0 = the launcher's model choice
    unsigned long long wait_ns;      // tensor-core kernels: bound of each device wait (0 = 2 s)
};
int zgemm_tile_count();              // number of SIMT tile candidates
int zgemm_model_tile(const GemmDesc &d);   // 1-based candidate the launcher's model picks
// Long-K GEMMs with few output tiles split K across CTAs (deterministic: partial sums go to
// `work`, then one reduction applies alpha / beta); work may be NULL (no split).
int zgemm_ksplit(const GemmDesc &d);
// split-K that fills whole waves of one CTA per SM for SIMT tile `tile` (1 = no split)
int zgemm_wave_split(const GemmDesc &d, int tile);
i64 zgemm_workspace_elems(const GemmDesc &d);   // split-K partials needed (0 without a split)
// returns the number of kernels launched
// few-row kernel (M <= 8, K nred <= 256): one thread per output column; returns 0 if not applicable
bool zgemm_smallm_supported(const GemmDesc &d);
template <typename R>
int launch_zgemm_smallm(const GemmDesc &d, const typename cvec<R>::T *A, const typename cvec<R>::T *B,
                        typename cvec<R>::T *C, cudaStream_t st);
template <typename R>
int launch_zgemm(const GemmDesc &d, const typename cvec<R>::T *A, const typename cvec<R>::T *B,
                 typename cvec<R>::T *C, cudaStream_t st, typename cvec<R>::T *work = nullptr, i64 work_elems = 0);

// ----------------------------------------------------------------------------- tensor GEMM
// C_b = alpha * sum_{r<nred} A_{b,r} B_{b,r} + beta * C_b where each GEMM index is a pair of tensor
// indices: index i sits at (i / d2) * s1 + (i % d2) * s2 of its operand (tgemm.cu).
struct IMap {
    int d2;
    i64 s1, s2;
};
IMap imap_single(i64 stride);                               // i -> i * stride
IMap imap_pair(int inner, i64 outer_stride, i64 inner_stride);   // i -> (i / inner, i % inner)
struct TGemm {
    int M, N, K, nred, batch;
    IMap am, ak, bk, bn, cm, cn;       // A[m, k], B[k, n], C[m, n]
    const i64 *offA, *offB, *offC;     // device tables: [batch * nred], [batch * nred], [batch]
    double2 alpha, beta;
};
// work: partial sums of the split over the contraction that a GEMM with few output tiles takes
// (tgemm_workspace_elems; NULL or too small: no split)
template <typename R>
int launch_tgemm(const TGemm &d, const typename cvec<R>::T *A, const typename cvec<R>::T *B, typename cvec<R>::T *C,
                 cudaStream_t st, typename cvec<R>::T *work = nullptr, i64 work_elems = 0);
// FP32 arithmetic on an FP64-stored A (rounded as it is loaded): operands without an FP32 copy
int launch_tgemm_a64(const TGemm &d, const double2 *A, const float2 *B, float2 *C, cudaStream_t st, float2 *work = nullptr,
                     i64 work_elems = 0);
int tgemm_ksplit(const TGemm &d);
i64 tgemm_workspace_elems(const TGemm &d);
struct GemmDesc;
TGemm tgemm_of(const GemmDesc &g);

// Host side of the build's tensor GEMMs: offset tables per call (kept until the caller clears
// `keep` after a synchronisation); every access is proven in bounds on the host before a launch.
i64 imap_span(const IMap &m, i64 dim);
struct ccgf_handle;
struct BuildGemm {
    ccgf_handle *h;
    cudaStream_t st;
    std::vector<DBuf<i64>> keep;
    ccgf_status run(const char *what, int M, int N, int K, int nred, IMap am, IMap ak, IMap bk, IMap bn, IMap cm, IMap cn,
                    const double2 *A, i64 lenA, const double2 *B, i64 lenB, double2 *C, i64 lenC, const std::vector<i64> &oA,
                    const std::vector<i64> &oB, const std::vector<i64> &oC, double alpha, double beta);
};

// ----------------------------------------------------------------------------- batched permute
// C[offC[b] + sum_d i_d sC_d] = alpha * A[offA[b] + sum_d i_d sA_d] + beta * C[...]
struct PermDesc {
    int nd;
    i64 dims[6];
    i64 sA[6], sC[6];
    i64 total;
    int batch;
    const i64 *offA, *offC;
    double2 alpha, beta;
};
// tcgen05 tensor-core path for FP32 operands (tc_gemm.cu): TF32 split, three MMAs per K-step;
// *err is set to 1 when a bounded wait gives up (C is then left unwritten by that CTA)
bool tc_zgemm_supported(const GemmDesc &d);
int launch_tc_zgemm(const GemmDesc &d, const float2 *A, const float2 *B, float2 *C, int *err, cudaStream_t st);
// the register-fed kernel on an FP64-stored A (an intermediate without an FP32 copy)
int launch_tc_zgemm_a64(const GemmDesc &d, const double2 *A, const float2 *B, float2 *C, int *err, cudaStream_t st);
struct ccgf_handle;
// TMA-fed variant: A = intermediate a_buf, read through tensor maps over its TF32 hi / lo copies
// (tc_prepare); rowA[b * nred + r] = offA / rsA. Returns 0 (nothing launched) when the shape or
// buffer does not qualify, else the number of launches.
int launch_tc_zgemm_tma(ccgf_handle *h, int a_buf, const GemmDesc &d, const i64 *rowA, const float2 *B, float2 *C, int *err,
                        cudaStream_t st);
// Bulk-fed variant: both operands by asynchronous copies; B' is first expanded into an image for
// the nslots distinct B blocks (bsrc[slot] = offset, bslot[b * nred + r] = slot).
int launch_tc_zgemm_bulk(ccgf_handle *h, int a_buf, const GemmDesc &d, const i64 *rowA, const i64 *bslot, const i64 *bsrc,
                         int nslots, const float2 *B, float2 *C, int *err, cudaStream_t st);
template <typename R>
int launch_zpermute(const PermDesc &d, const typename cvec<R>::T *A, typename cvec<R>::T *C, cudaStream_t st);

// ----------------------------------------------------------------------------- k-mesh
struct KMeshH {
    int n[3];
    int nk;
    std::vector<int> add, sub;   // add[a*nk+b] = a+b, sub[a*nk+b] = a-b
    void init(const int kmesh[3]);
    int a(int x, int y) const { return add[x * nk + y]; }
    int s(int x, int y) const { return sub[x * nk + y]; }
    int c(int k1, int k2, int k3) const { return a(s(k1, k2), k3); }   // k1 - k2 + k3
};

// ----------------------------------------------------------------------------- sigma plan
// A sigma plan is a list of launches over fixed buffers: A operands are
// intermediates (buffer ids below), B operands always live in the scratch arena
// (the input vector is copied there first), C operands are the output or scratch.
enum { STEP_GEMM = 0, STEP_PERM = 1, STEP_FOV_IP = 2, STEP_FOV_EA = 3, STEP_LADDER_GATHER = 4, STEP_LADDER_SCATTER = 5,
       STEP_TGEMM = 6 };
struct SigmaStep {
    const char *name;
    int kind;
    GemmDesc g;
    PermDesc p;
    TGemm tg;          // STEP_TGEMM: tensor GEMM; operands a_buf, b_buf, c_buf (intermediate, BUF_SCRATCH or BUF_Y)
    int b_buf;
    int a_buf;         // GEMM: intermediate id (or BUF_SCRATCH); PERM: source (BUF_SCRATCH)
    int c_buf;         // BUF_Y or BUF_SCRATCH
    i64 offA_pos, offB_pos, offC_pos;   // positions in the plan's offset table
    i64 lad_rp, lad_rm;                 // ladder gather / scatter: scratch offsets of R+ / S+ and R- / S-
    i64 rowA_pos;                       // GEMM: position of offA / rsA per (batch, reduction), -1 if not integral
    i64 bslot_pos, bsrc_pos;            // GEMM: slot of each (batch, reduction) B block, offsets of the distinct blocks
    int nslots;                         // number of distinct B blocks
    int choice[4];                      // GEMM kernel measured per precision index (0 = not tuned; see sigma.cu)
};
struct SigmaPlan {
    int sector, K, nv;
    std::vector<SigmaStep> steps;
    DBuf<i64> offsets;
    std::vector<i64> host_off;
    i64 scratch_elems;
    i64 seg[12];       // scratch segment offsets (complex elements)
};

enum {
    BUF_Y = 0, BUF_SCRATCH,
    BUF_FOO, BUF_FVV, BUF_FOV,
    BUF_WVVVV, BUF_WPLUS, BUF_WMINUS, BUF_WVVVO, BUF_WOV3, BUF_UVOVV, BUF_UOOVV_EA, BUF_T2EA,
    BUF_WOVOO, BUF_WOOOO, BUF_UOOOV, BUF_UOOVV_IP, BUF_T2IP,
    // operands of the terms evaluated from the density-fitting factors (tensor GEMMs):
    // dressed factors L~[k1][k2][Q][p][q], the <mn|ef> block (m e | n f)[km][ke][kn][m][e][n][f], T2
    BUF_LD, BUF_OVOV, BUF_T2,
    NBUF
};

struct WarmStart;
struct ccgf_handle {
    // true: the W_vvvo r1 term, the (2<am|ef> - <am|fe>) r2 term of the EA singles and the T2 part of
    // the EA ladder are evaluated in every sigma from the density-fitting factors instead of being
    // stored (the memory-scalable form for large k-meshes and virtual spaces)
    bool direct = false;
    int device;
    KMeshH km;
    int nk, o, v, n, naux;
    i64 dim_ip, dim_ea;
    // FP64 inputs kept on device
    DBuf<double2> t1, t2, l1, l2, L;
    DBuf<double> eps;
    DBuf<int> kadd_d, ksub_d;   // momentum tables on device
    // FP64 intermediates (GEMM-ready), FP32 copies below
    DBuf<double2> W[NBUF];
    DBuf<float2> Wf[NBUF];
    bool fp32_done = false;   // FP32 copies decided (a block may stay FP64-only for lack of memory)
    i64 wov_seg;       // size of each of W1 | W2 | WN inside BUF_WOV3
    // pair-symmetric EA ladder: representatives per pair momentum and padded block sizes
    std::vector<int> lad_np, lad_nm;
    int lad_Pp = 0, lad_Pm = 0;
    DBuf<int> lad_reps, lad_npl, lad_nmi;
    // scratch arena for sigma (FP64 and FP32 variants) and the FP32 output
    DBuf<double2> scratch;
    DBuf<float2> scratch_f, yf;
    // split-K workspaces of the autotuner's wave-filling splits (grown on demand)
    DBuf<double2> splitw64;
    DBuf<float2> splitw32;
    // error flag of the tensor-core GEMMs and their TF32-split operands (made on first CCGF_TF32X3 use)
    DBuf<int> tc_err;
    void *tc_ops = nullptr;
    // FP64-accurate tensor-core path (tc_gemm.cu): sliced planes of the intermediates, made on first use
    // only while oz_reserve bytes of device memory stay free
    void *oz_ops = nullptr;
    size_t oz_reserve = (size_t)4 << 30;
    // cached plans, index (sector-1)*nk + K, valid for plan_nv columns
    std::vector<SigmaPlan *> plans;
    int plan_nv = 0;
    i64 launches = 0;
    // learned warm start (mlp.cu); capture of training solutions while ws_capturing
    WarmStart *ws = nullptr;
    // model-order reduction (mor.cu): solutions of one (sector, K) kept as columns p * ncols_w + w
    struct MorCapture {
        int sector = 0, K = -1, nw = 0;
        double2 *X = nullptr;   // [D][nmo * nw]
    } mor_cap;
    bool ws_capturing = false;
    // right-hand sides b_p and left vectors e_q of solve_gf per (sector, K) (they do not depend on the
    // frequency), kept while their total stays under a small share of device memory
    struct VecCache {
        DBuf<double2> Bq, E;
    };
    std::vector<VecCache *> vcache;
    size_t vcache_bytes = 0;
    // bound of every tensor-core device wait (from ccgf_options::device_wait_timeout_ms)
    unsigned long long wait_ns = 1000000000ull;
    // three zero offsets on this handle's device (single-block GEMM / permute launches)
    DBuf<i64> zero_tab;
    // layout transposes of ccgf_sigma_ip / ea (grown on demand, reused across calls)
    DBuf<double2> abi_x, abi_y;
    // optional per-step timing of one sigma call (ccgf_sigma_profile)
    cudaEvent_t *prof_events = nullptr;
    int prof_max = 0, prof_count = 0;
};

// build.cu
ccgf_status build_intermediates(ccgf_handle *h, const ccgf_system *sys, const ccgf_options *opt, cudaStream_t st);
// sigma.cu: W_vvvo[K] (stored form) = the EA r1 -> r2 terms applied to unit vectors, for every K
ccgf_status build_wvvvo_by_plan(ccgf_handle *h, cudaStream_t st);
// sigma.cu
double plan_step_flops(const ccgf_handle *h, int sector, int K, int step);   // algorithmic flops of a plan step
int plan_step_count(const ccgf_handle *h, int sector, int K);
const char *plan_step_name(const ccgf_handle *h, int sector, int K, int step);
ccgf_status sigma_apply(ccgf_handle *h, int sector, int K, int nv, const double2 *x, double2 *y,
                        ccgf_precision prec, cudaStream_t st);
void free_plans(ccgf_handle *h);
void release_caches(ccgf_handle *h);   // FP32 / TF32 copies, scratch arenas (rebuilt on demand)
void vcache_free(ccgf_handle *h);      // solve.cu: cached right-hand sides and left vectors
void set_autotune(bool on);
int plan_step_choice(const ccgf_handle *h, int sector, int K, int step, int prec_index);
// reads and clears the tensor-core error flag (synchronises st); CCGF_ERR_TIMEOUT when it was set
ccgf_status tc_error_check(ccgf_handle *h, cudaStream_t st);
// tc_gemm.cu: the bounded-wait timeout path alone (one warp, a barrier nothing arrives on)
void launch_wait_selftest(double limit_ms, int *err, cudaStream_t st);
// tc_gemm.cu: TF32 hi / lo copies of every FP32 intermediate, freed by tc_free
// (only for blocks with an FP32 copy, and only while `reserve` bytes of device memory stay free)
ccgf_status tc_prepare(ccgf_handle *h, cudaStream_t st, size_t reserve);
// FP64-accurate complex GEMM on the tensor cores (sliced operands; C and B FP64, A a stored intermediate
// with TMA-addressable rows): returns launches, 0 when the shape, the tables or device memory do not allow it
bool tc_zgemm_oz_supported(const GemmDesc &d);
int launch_tc_zgemm_oz(ccgf_handle *h, int a_buf, const GemmDesc &d, const i64 *rowA, const i64 *bslot, const i64 *bsrc, int nslots,
                       const double2 *B, double2 *C, int *err, cudaStream_t st);
void oz_free(ccgf_handle *h);
// sigma.cu: FP32 copies of the intermediates (large blocks only while `reserve` bytes stay free)
ccgf_status ensure_fp32(ccgf_handle *h, cudaStream_t st, size_t reserve);
void tc_free(ccgf_handle *h);
ccgf_status sigma_apply_in_arena(ccgf_handle *h, int sector, int K, int nv, const double2 *x, double2 *y, double2 *arena,
                                 i64 arena_elems, i64 *offsets, i64 offsets_cap, cudaStream_t st);
i64 sigma_arena_elems(const ccgf_handle *h, int nv);
i64 sigma_scratch_per_column(const ccgf_handle *h);
// vectors.cu
ccgf_status make_rhs(ccgf_handle *h, int sector, int K, int p, double2 *out, i64 ld, cudaStream_t st);
ccgf_status make_left(ccgf_handle *h, int sector, int K, int p, double2 *out, i64 ld, cudaStream_t st);
// transposes between [nvec][D] (ABI) and [D][nv] (internal)
void launch_transpose_in(const double2 *x, double2 *xt, i64 D, int nvec, int nv, cudaStream_t st);
void launch_transpose_out(const double2 *yt, double2 *y, i64 D, int nvec, int nv, cudaStream_t st);
// mlp.cu
ccgf_status warmstart_begin_capture(ccgf_handle *h, const double *omega, int n, double eta);
ccgf_status warmstart_capture(ccgf_handle *h, int sector, int K, const double2 *X, i64 D, int nw, int w0, const double *bnorm2_h,
                              cudaStream_t st);
// x0 of the network into X; when the learned correction is in use, the baseline alone into Xbase
ccgf_status warmstart_infer(ccgf_handle *h, int sector, int K, const double *om, int nw, const double *dvec, double2 *X,
                            double2 *Xbase, bool *used, bool *net, cudaStream_t st);
ccgf_status warmstart_train(ccgf_handle *h, int sectors, int steps, i64 rows, double lr, unsigned seed, double *final_loss,
                            cudaStream_t st);
void warmstart_free(ccgf_handle *h);
void warmstart_losses(const ccgf_handle *h, double *val_net, double *val_base);
// solve.cu: copies the converged columns of one batch into the model-order-reduction capture
void mor_capture_columns(ccgf_handle *h, const double2 *X, i64 D, int nv, int p0, int pend, int nw, int w0, cudaStream_t st);
// solve.cu
ccgf_status diag_estimate_device(ccgf_handle *h, int sector, int K, double *d, cudaStream_t st);
ccgf_status solve_gf_mor(ccgf_handle *h, int sectors, int n_mor, const double *omega_mor, int nomega, const double *omega,
                         double eta, const ccgf_options *opt, double *G_out, int G_on_device, ccgf_stats *stats, cudaStream_t st);
ccgf_status solve_gf(ccgf_handle *h, int sectors, int nomega, const double *omega, double eta,
                     const ccgf_options *opt, double *G_out, int G_on_device, ccgf_stats *stats,
                     cudaStream_t st);

inline i64 ceil_div(i64 a, i64 b) { return (a + b - 1) / b; }
