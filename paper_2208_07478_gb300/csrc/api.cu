// extern "C" entry points of the CCGF library (see include/ccgf.h).
#include "ccgf_internal.h"
#include <cmath>
#include <new>
#include <vector>

namespace {

ccgf_status copy_in(DBuf<double2> &dst, const double *src, i64 n, bool on_device, cudaStream_t st) {
    CCGF_TRY(dalloc(dst, n));
    CCGF_CUDA_TRY(cudaMemcpyAsync(dst.p, src, sizeof(double2) * n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    return CCGF_OK;
}

__global__ void conj_kernel(const double2 *a, double2 *b, i64 n) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) b[i] = make_double2(a[i].x, -a[i].y);
}

bool valid_wait(double ms) { return ms > 0.0 && ms <= 60000.0; }
unsigned long long wait_ns_of(double ms) { return (unsigned long long)(ms * 1e6); }

void destroy(ccgf_handle *h) {
    if (!h) return;
    warmstart_free(h);
    free_plans(h);
    dfree(h->t1);
    dfree(h->t2);
    dfree(h->l1);
    dfree(h->l2);
    dfree(h->L);
    dfree(h->eps);
    dfree(h->kadd_d);
    dfree(h->ksub_d);
    dfree(h->lad_reps);
    dfree(h->lad_npl);
    dfree(h->lad_nmi);
    for (int b = 0; b < NBUF; ++b) {
        dfree(h->W[b]);
        dfree(h->Wf[b]);
    }
    dfree(h->scratch);
    dfree(h->scratch_f);
    dfree(h->yf);
    dfree(h->tc_err);
    dfree(h->splitw64);
    dfree(h->splitw32);
    dfree(h->zero_tab);
    dfree(h->abi_x);
    dfree(h->abi_y);
    tc_free(h);
    oz_free(h);
    vcache_free(h);
    delete h;
}

}  // namespace

extern "C" {

void ccgf_default_options(ccgf_options *opt) {
    if (!opt) return;
    opt->prec = CCGF_FP64;
    opt->tol = 1e-10;
    opt->restart_m = 30;
    opt->max_iter = 2000;
    opt->max_refine = 20;
    opt->omega_chunk = 1;
    opt->device_wait_timeout_ms = 1000.0;
    opt->warm_start = 0;
    opt->kpoint = -1;
    opt->orbital_first = 0;
    opt->orbital_count = 0;
    opt->direct_terms = 0;
    opt->refine_prec = CCGF_FP64;
}

const char *ccgf_status_string(ccgf_status s) {
    switch (s) {
        case CCGF_OK: return "ok";
        case CCGF_NOT_CONVERGED: return "not converged (outputs written)";
        case CCGF_ERR_INVALID_ARG: return "invalid argument";
        case CCGF_ERR_OOM: return "out of device memory";
        case CCGF_ERR_CUDA: return "CUDA error";
        case CCGF_ERR_NAN: return "non-finite input";
        case CCGF_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

ccgf_status ccgf_build_intermediates(const ccgf_system *sys, const ccgf_options *opt, void *stream, ccgf_handle **out) {
    if (!sys || !out) { set_last_error("NULL system or output pointer"); return CCGF_ERR_INVALID_ARG; }
    if (opt && !valid_wait(opt->device_wait_timeout_ms)) {
        set_last_error("device_wait_timeout_ms must be in (0, 60000]");
        return CCGF_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (sys->kmesh[0] < 1 || sys->kmesh[1] < 1 || sys->kmesh[2] < 1 || sys->nocc < 1 || sys->nvir < 1 || sys->naux < 1) {
        set_last_error("kmesh, nocc, nvir and naux must be >= 1");
        return CCGF_ERR_INVALID_ARG;
    }
    if (!sys->mo_energy || !sys->L || !sys->t1 || !sys->t2) { set_last_error("NULL input array"); return CCGF_ERR_INVALID_ARG; }
    ccgf_handle *h = new (std::nothrow) ccgf_handle();
    if (!h) { set_last_error("host allocation failed"); return CCGF_ERR_OOM; }
    cudaStream_t st = (cudaStream_t)stream;
    cudaGetDevice(&h->device);
    if (opt) h->wait_ns = wait_ns_of(opt->device_wait_timeout_ms);
    h->km.init(sys->kmesh);
    h->nk = h->km.nk;
    h->o = sys->nocc;
    h->v = sys->nvir;
    h->n = sys->nocc + sys->nvir;
    h->naux = sys->naux;
    const i64 nk = h->nk, o = h->o, v = h->v, n = h->n;
    h->dim_ip = o + nk * nk * o * o * v;
    h->dim_ea = v + nk * nk * o * v * v;
    const bool dev = sys->inputs_on_device != 0;
    ccgf_status s = CCGF_OK;
    auto fail = [&](ccgf_status e) { destroy(h); return e; };
    if ((s = copy_in(h->L, sys->L, nk * nk * h->naux * n * n, dev, st)) != CCGF_OK) return fail(s);
    if ((s = copy_in(h->t1, sys->t1, nk * o * v, dev, st)) != CCGF_OK) return fail(s);
    if ((s = copy_in(h->t2, sys->t2, nk * nk * nk * o * o * v * v, dev, st)) != CCGF_OK) return fail(s);
    if ((s = dalloc(h->eps, nk * n)) != CCGF_OK) return fail(s);
    if (cudaMemcpyAsync(h->eps.p, sys->mo_energy, sizeof(double) * nk * n, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st) != cudaSuccess) {
        set_last_error("copy of mo_energy failed");
        return fail(CCGF_ERR_CUDA);
    }
    if (sys->l1) {
        if ((s = copy_in(h->l1, sys->l1, nk * o * v, dev, st)) != CCGF_OK) return fail(s);
    } else {
        if ((s = dalloc(h->l1, nk * o * v)) != CCGF_OK) return fail(s);
        conj_kernel<<<256, 256, 0, st>>>(h->t1.p, h->l1.p, h->l1.n);
        h->launches++;
    }
    if (sys->l2) {
        if ((s = copy_in(h->l2, sys->l2, h->t2.n, dev, st)) != CCGF_OK) return fail(s);
    } else {
        if ((s = dalloc(h->l2, h->t2.n)) != CCGF_OK) return fail(s);
        conj_kernel<<<1024, 256, 0, st>>>(h->t2.p, h->l2.p, h->l2.n);
        h->launches++;
    }
    if ((s = build_intermediates(h, sys, opt, st)) != CCGF_OK) return fail(s);
    *out = h;
    return CCGF_OK;
}

ccgf_status ccgf_dims(const ccgf_handle *h, int *nk, int *nocc, int *nvir, long long *dim_ip, long long *dim_ea) {
    if (!h) { set_last_error("NULL handle"); return CCGF_ERR_INVALID_ARG; }
    if (nk) *nk = h->nk;
    if (nocc) *nocc = h->o;
    if (nvir) *nvir = h->v;
    if (dim_ip) *dim_ip = h->dim_ip;
    if (dim_ea) *dim_ea = h->dim_ea;
    return CCGF_OK;
}

static bool valid_prec(ccgf_precision p) {
    return p == CCGF_FP64 || p == CCGF_FP32 || p == CCGF_TF32X3 || p == CCGF_FP64_TC;
}

static ccgf_status sigma_abi(ccgf_handle *h, int sector, int kshift, long long nvec, const double *x, double *y,
                             ccgf_precision prec, void *stream) {
    if (!h || !x || !y) { set_last_error("NULL handle or vector"); return CCGF_ERR_INVALID_ARG; }
    if (kshift < 0 || kshift >= h->nk) { set_last_error("kshift out of range"); return CCGF_ERR_INVALID_ARG; }
    if (nvec < 1 || nvec > 65536) { set_last_error("nvec must be in [1, 65536]"); return CCGF_ERR_INVALID_ARG; }
    if (!valid_prec(prec)) { set_last_error("unknown precision"); return CCGF_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const i64 D = sector == CCGF_SECTOR_IP ? h->dim_ip : h->dim_ea;
    const int nv = (int)nvec;
    if (h->abi_x.n < D * nv) {
        // grow the handle's transpose buffers (cudaFree waits for work that may still read them)
        CCGF_TRY(dalloc(h->abi_x, D * nv));
        CCGF_TRY(dalloc(h->abi_y, D * nv));
    }
    launch_transpose_in((const double2 *)x, h->abi_x.p, D, nv, nv, st);
    CCGF_TRY(sigma_apply(h, sector, kshift, nv, h->abi_x.p, h->abi_y.p, prec, st));
    launch_transpose_out(h->abi_y.p, (double2 *)y, D, nv, nv, st);
    h->launches += 2;
    CCGF_CUDA_TRY(cudaGetLastError());
    if (prec == CCGF_TF32X3 || prec == CCGF_FP64_TC) return tc_error_check(h, st);
    return CCGF_OK;
}

ccgf_status ccgf_sigma_ip(ccgf_handle *h, int kshift, long long nvec, const double *x, double *y, ccgf_precision prec, void *stream) {
    return sigma_abi(h, CCGF_SECTOR_IP, kshift, nvec, x, y, prec, stream);
}
ccgf_status ccgf_sigma_ea(ccgf_handle *h, int kshift, long long nvec, const double *x, double *y, ccgf_precision prec, void *stream) {
    return sigma_abi(h, CCGF_SECTOR_EA, kshift, nvec, x, y, prec, stream);
}

static ccgf_status vec_abi(ccgf_handle *h, int sector, int K, int p, double *out, void *stream, bool left) {
    if (!h || !out) { set_last_error("NULL handle or output"); return CCGF_ERR_INVALID_ARG; }
    if (sector != CCGF_SECTOR_IP && sector != CCGF_SECTOR_EA) { set_last_error("sector must be IP or EA"); return CCGF_ERR_INVALID_ARG; }
    if (K < 0 || K >= h->nk || p < 0 || p >= h->n) { set_last_error("K or orbital out of range"); return CCGF_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    ccgf_status s = left ? make_left(h, sector, K, p, (double2 *)out, 1, st) : make_rhs(h, sector, K, p, (double2 *)out, 1, st);
    if (s != CCGF_OK) return s;
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    return CCGF_OK;
}
ccgf_status ccgf_rhs(ccgf_handle *h, int sector, int K, int p, double *out, void *stream) { return vec_abi(h, sector, K, p, out, stream, false); }
ccgf_status ccgf_left(ccgf_handle *h, int sector, int K, int p, double *out, void *stream) { return vec_abi(h, sector, K, p, out, stream, true); }

ccgf_status ccgf_solve_gf(ccgf_handle *h, int sectors, int nomega, const double *omega, double eta, const ccgf_options *opt,
                          double *G_out, int G_on_device, ccgf_stats *stats, void *stream) {
    if (!h || !omega || !G_out) { set_last_error("NULL handle, omega or output"); return CCGF_ERR_INVALID_ARG; }
    if (sectors < 1 || sectors > 3 || nomega < 1) { set_last_error("sectors must be 1..3 and nomega >= 1"); return CCGF_ERR_INVALID_ARG; }
    if (!(eta > 0.0) || !std::isfinite(eta)) { set_last_error("eta must be positive and finite"); return CCGF_ERR_INVALID_ARG; }
    for (int w = 0; w < nomega; ++w)
        if (!std::isfinite(omega[w])) { set_last_error("non-finite frequency"); return CCGF_ERR_NAN; }
    ccgf_options o;
    if (opt) o = *opt;
    else ccgf_default_options(&o);
    if (!(o.tol > 0.0) || o.restart_m < 2 || o.max_iter < 1 || o.max_refine < 1 || o.omega_chunk < 1) {
        set_last_error("invalid options (tol > 0, restart_m >= 2, max_iter >= 1, max_refine >= 1, omega_chunk >= 1)");
        return CCGF_ERR_INVALID_ARG;
    }
    if (!valid_prec(o.prec) || (o.refine_prec != CCGF_FP64 && o.refine_prec != CCGF_FP64_TC)) { set_last_error("unknown precision"); return CCGF_ERR_INVALID_ARG; }
    if (!valid_wait(o.device_wait_timeout_ms)) { set_last_error("device_wait_timeout_ms must be in (0, 60000]"); return CCGF_ERR_INVALID_ARG; }
    if (o.kpoint < -1 || o.kpoint >= h->nk || o.orbital_first < 0 || o.orbital_count < 0 ||
        o.orbital_first + o.orbital_count > h->n || (o.orbital_count == 0 && o.orbital_first != 0)) {
        set_last_error("kpoint must be -1 or a k index; orbital_first / orbital_count must select orbitals of the cell");
        return CCGF_ERR_INVALID_ARG;
    }
    // the solve's own wait bound for its duration; the handle's build-time bound afterwards
    struct WaitScope {
        ccgf_handle *h;
        unsigned long long saved;
        ~WaitScope() { h->wait_ns = saved; }
    } scope{h, h->wait_ns};
    h->wait_ns = wait_ns_of(o.device_wait_timeout_ms);
    return solve_gf(h, sectors, nomega, omega, eta, &o, G_out, G_on_device, stats, (cudaStream_t)stream);
}

ccgf_status ccgf_solve_gf_mor(ccgf_handle *h, int sectors, int n_mor, const double *omega_mor, int nomega, const double *omega,
                              double eta, const ccgf_options *opt, double *G_out, int G_on_device, ccgf_stats *stats, void *stream) {
    if (!h || !omega || !omega_mor || !G_out) { set_last_error("NULL handle, frequencies or output"); return CCGF_ERR_INVALID_ARG; }
    if (sectors < 1 || sectors > 3 || nomega < 1 || n_mor < 1 || n_mor > 64) {
        set_last_error("sectors must be 1..3, nomega >= 1 and 1 <= n_mor <= 64");
        return CCGF_ERR_INVALID_ARG;
    }
    if (!(eta > 0.0) || !std::isfinite(eta)) { set_last_error("eta must be positive and finite"); return CCGF_ERR_INVALID_ARG; }
    for (int w = 0; w < nomega; ++w)
        if (!std::isfinite(omega[w])) { set_last_error("non-finite frequency"); return CCGF_ERR_NAN; }
    for (int w = 0; w < n_mor; ++w)
        if (!std::isfinite(omega_mor[w])) { set_last_error("non-finite model frequency"); return CCGF_ERR_NAN; }
    ccgf_options o;
    if (opt) o = *opt;
    else ccgf_default_options(&o);
    if (!(o.tol > 0.0) || o.restart_m < 2 || o.max_iter < 1 || o.max_refine < 1 || o.omega_chunk < 1 || o.kpoint < -1 ||
        o.kpoint >= h->nk || !valid_wait(o.device_wait_timeout_ms)) {
        set_last_error("invalid options");
        return CCGF_ERR_INVALID_ARG;
    }
    if (!valid_prec(o.prec) || (o.refine_prec != CCGF_FP64 && o.refine_prec != CCGF_FP64_TC)) { set_last_error("unknown precision"); return CCGF_ERR_INVALID_ARG; }
    struct WaitScope {
        ccgf_handle *h;
        unsigned long long saved;
        ~WaitScope() { h->wait_ns = saved; }
    } scope{h, h->wait_ns};
    h->wait_ns = wait_ns_of(o.device_wait_timeout_ms);
    return solve_gf_mor(h, sectors, n_mor, omega_mor, nomega, omega, eta, &o, G_out, G_on_device, stats, (cudaStream_t)stream);
}

ccgf_status ccgf_sigma_profile(ccgf_handle *h, int sector, int kshift, long long nvec, const double *x, double *y,
                               ccgf_precision prec, void *stream, int max_steps, double *step_ms, double *step_flops,
                               int *nsteps) {
    if (!h || !step_ms || !step_flops || !nsteps || max_steps < 1) { set_last_error("NULL output or max_steps < 1"); return CCGF_ERR_INVALID_ARG; }
    if (sector != CCGF_SECTOR_IP && sector != CCGF_SECTOR_EA) { set_last_error("sector must be IP or EA"); return CCGF_ERR_INVALID_ARG; }
    std::vector<cudaEvent_t> ev(max_steps + 1, nullptr);
    auto cleanup = on_scope_exit([&] {
        h->prof_events = nullptr;
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    });
    for (auto &e : ev) CCGF_CUDA_TRY(cudaEventCreate(&e));
    h->prof_events = ev.data();
    h->prof_max = max_steps + 1;
    h->prof_count = 0;
    ccgf_status s = sigma_abi(h, sector, kshift, nvec, x, y, prec, stream);
    if (s == CCGF_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        set_last_error("stream synchronisation after the profiled sigma failed");
        s = CCGF_ERR_CUDA;
    }
    h->prof_events = nullptr;
    int n = plan_step_count(h, sector, kshift);
    *nsteps = n;
    if (s == CCGF_OK) {
        for (int i = 0; i < n && i < max_steps; ++i) {
            float ms = 0.f;
            if (i + 1 < h->prof_count) cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            step_ms[i] = ms;
            step_flops[i] = plan_step_flops(h, sector, kshift, i);
        }
    }
    return s;
}

const char *ccgf_sigma_step_name(const ccgf_handle *h, int sector, int kshift, int step) {
    return h ? plan_step_name(h, sector, kshift, step) : "";
}

long long ccgf_launch_count(const ccgf_handle *h) { return h ? h->launches : 0; }

void ccgf_set_autotune(int enable) { set_autotune(enable != 0); }

ccgf_status ccgf_tensor_wait_selftest(double limit_ms, void *stream) {
    if (!(limit_ms > 0.0) || limit_ms > 2000.0) { set_last_error("limit_ms must be in (0, 2000]"); return CCGF_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    DBuf<int> flag;
    CCGF_TRY(dalloc(flag, 1));
    CCGF_CUDA_TRY(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    launch_wait_selftest(limit_ms, flag.p, st);
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(flag);
    if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); return CCGF_ERR_CUDA; }
    if (v) {
        set_last_error("tensor-core wait self-test: the wait gave up after its limit, as designed");
        return CCGF_ERR_TIMEOUT;
    }
    return CCGF_OK;
}
int ccgf_sigma_step_kernel(const ccgf_handle *h, int sector, int kshift, int step, ccgf_precision prec) {
    if (!h || !valid_prec(prec)) return -1;
    return plan_step_choice(h, sector, kshift, step, (int)prec);
}

ccgf_status ccgf_train_warmstart(ccgf_handle *h, int sectors, int n_train, const double *omega_train, double eta,
                                 const ccgf_options *opt, int steps, long long rows_per_step, double lr, unsigned seed,
                                 double *final_loss, ccgf_stats *stats, void *stream) {
    if (!h || !omega_train || n_train < 3 || sectors < 1 || sectors > 3 || steps < 0 || rows_per_step < 64 ||
        rows_per_step > (1LL << 22) || !(lr > 0) || !(eta > 0)) {
        set_last_error("invalid warm-start training arguments (n_train >= 3, steps >= 0, 64 <= rows <= 4M, lr, eta > 0)");
        return CCGF_ERR_INVALID_ARG;
    }
    for (int i = 1; i < n_train; ++i)
        if (!(omega_train[i] > omega_train[i - 1])) { set_last_error("training frequencies must increase"); return CCGF_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    ccgf_options o;
    if (opt) o = *opt;
    else ccgf_default_options(&o);
    o.warm_start = 0;
    CCGF_TRY(warmstart_begin_capture(h, omega_train, n_train, eta));
    const i64 Gn = (i64)h->nk * n_train * h->n * h->n;
    DBuf<double2> G;
    CCGF_TRY(dalloc(G, Gn));
    h->ws_capturing = true;
    ccgf_status s = solve_gf(h, sectors, n_train, omega_train, eta, &o, (double *)G.p, 1, stats, st);
    h->ws_capturing = false;
    dfree(G);
    if (s != CCGF_OK && s != CCGF_NOT_CONVERGED) return s;
    s = warmstart_train(h, sectors, steps, rows_per_step, lr, seed, final_loss, st);
    if (s == CCGF_OK && stats) warmstart_losses(h, &stats->warm_val_loss, &stats->warm_val_loss_baseline);
    return s;
}

void ccgf_destroy(ccgf_handle *h) { destroy(h); }

}  // extern "C"
