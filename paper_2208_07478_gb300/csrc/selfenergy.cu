// Active-space self-energy correction (Eqs. 12-14): with natural-orbital coefficients V(k) (N x M,
// the M active orbitals in the N-orbital basis), the coupled-cluster G of the active space and the
// GW Green's functions of the full space and of the active space,
//   Sigma_CAS  = G_GW,CAS^-1 - G_CC,CAS^-1                  (M x M)      Eq. 12
//   Sigma_full = V Sigma_CAS V^+                            (N x N)      Eq. 13
//   G_CC+GW    = [G_GW,full^-1 - Sigma_full]^-1             (N x N)      Eq. 14
// for every (k, w). One thread block per (k, w): Gauss-Jordan inversions with partial pivoting in
// shared memory, the products in shared memory as well.
#include "ccgf_internal.h"

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// in-place inverse of the n x n matrix a (row-major, shared memory); piv: n ints; returns false if singular
__device__ bool gj_inverse(double2 *a, int n, int *piv, double2 *col, int *bad) {
    const int t = threadIdx.x, nt = blockDim.x;
    for (int k = 0; k < n; ++k) {
        if (t == 0) {
            int best = k;
            double bm = -1.0;
            for (int i = k; i < n; ++i) {
                const double m = fabs(a[i * n + k].x) + fabs(a[i * n + k].y);
                if (m > bm) { bm = m; best = i; }
            }
            piv[k] = best;
            if (!(bm > 0.0)) *bad = 1;
        }
        __syncthreads();
        if (*bad) return false;
        const int p = piv[k];
        if (p != k)
            for (int j = t; j < n; j += nt) {
                const double2 tmp = a[k * n + j];
                a[k * n + j] = a[p * n + j];
                a[p * n + j] = tmp;
            }
        __syncthreads();
        const double2 d = a[k * n + k];
        for (int i = t; i < n; i += nt) col[i] = a[i * n + k];
        __syncthreads();
        // row k /= d (the pivot column becomes 1 / d); other rows i -= col[i] * row k
        for (int j = t; j < n; j += nt) a[k * n + j] = j == k ? cdiv(make_double2(1, 0), d) : cdiv(a[k * n + j], d);
        __syncthreads();
        for (int e = t; e < n * n; e += nt) {
            const int i = e / n, j = e % n;
            if (i == k) continue;
            const double2 rk = a[k * n + j];
            double2 v = j == k ? make_double2(0, 0) : a[i * n + j];
            const double2 pr = cmul(col[i], rk);
            a[i * n + j] = make_double2(v.x - pr.x, v.y - pr.y);
        }
        __syncthreads();
    }
    // undo the row exchanges as column exchanges of the inverse, last first
    for (int k = n - 1; k >= 0; --k) {
        const int p = piv[k];
        if (p != k)
            for (int i = t; i < n; i += nt) {
                const double2 tmp = a[i * n + k];
                a[i * n + k] = a[i * n + p];
                a[i * n + p] = tmp;
            }
        __syncthreads();
    }
    return true;
}

__global__ void self_energy_kernel(int nomega, int N, int M, const double2 *__restrict__ V, const double2 *__restrict__ Ggw,
                                   const double2 *__restrict__ Ggw_cas, const double2 *__restrict__ Gcc_cas, double2 *Gout,
                                   int *err) {
    extern __shared__ double2 sm[];
    double2 *sA = sm;                   // N x N
    double2 *sS = sA + N * N;           // M x M (Sigma_CAS)
    double2 *sT = sS + M * M;           // M x M, then N x M
    double2 *col = sT + N * M + M * M;  // N
    int *piv = (int *)(col + N);        // N
    __shared__ int bad;
    const int t = threadIdx.x, nt = blockDim.x;
    const i64 kw = blockIdx.x;
    const int k = (int)(kw / nomega);
    const double2 *Vk = V + (i64)k * N * M;
    if (t == 0) bad = 0;
    // Sigma_CAS = G_GW,CAS^-1 - G_CC,CAS^-1
    for (int e = t; e < M * M; e += nt) sS[e] = Ggw_cas[kw * M * M + e];
    __syncthreads();
    if (!gj_inverse(sS, M, piv, col, &bad)) { if (t == 0) atomicExch(err, 1); return; }
    for (int e = t; e < M * M; e += nt) sT[e] = Gcc_cas[kw * M * M + e];
    __syncthreads();
    if (!gj_inverse(sT, M, piv, col, &bad)) { if (t == 0) atomicExch(err, 1); return; }
    for (int e = t; e < M * M; e += nt) sS[e] = make_double2(sS[e].x - sT[e].x, sS[e].y - sT[e].y);
    __syncthreads();
    // T = V Sigma_CAS (N x M)
    double2 *sVS = sT + M * M;
    for (int e = t; e < N * M; e += nt) {
        const int i = e / M, j = e % M;
        double2 acc = make_double2(0, 0);
        for (int l = 0; l < M; ++l) {
            const double2 p = cmul(Vk[(i64)i * M + l], sS[l * M + j]);
            acc.x += p.x;
            acc.y += p.y;
        }
        sVS[e] = acc;
    }
    // A = G_GW,full^-1
    for (int e = t; e < N * N; e += nt) sA[e] = Ggw[kw * N * N + e];
    __syncthreads();
    if (!gj_inverse(sA, N, piv, col, &bad)) { if (t == 0) atomicExch(err, 1); return; }
    // A -= (V Sigma_CAS) V^+
    for (int e = t; e < N * N; e += nt) {
        const int i = e / N, j = e % N;
        double2 acc = make_double2(0, 0);
        for (int l = 0; l < M; ++l) {
            const double2 vv = Vk[(i64)j * M + l];
            const double2 p = cmul(sVS[i * M + l], make_double2(vv.x, -vv.y));
            acc.x += p.x;
            acc.y += p.y;
        }
        sA[e] = make_double2(sA[e].x - acc.x, sA[e].y - acc.y);
    }
    __syncthreads();
    if (!gj_inverse(sA, N, piv, col, &bad)) { if (t == 0) atomicExch(err, 1); return; }
    for (int e = t; e < N * N; e += nt) Gout[kw * N * N + e] = sA[e];
}

}  // namespace

extern "C" ccgf_status ccgf_self_energy_correction(int nk, int nomega, int nmo, int nact, const double *V, const double *G_gw,
                                                   const double *G_gw_cas, const double *G_cc_cas, double *G_out, void *stream) {
    if (nk < 1 || nomega < 1 || nmo < 1 || nact < 1 || nact > nmo || !V || !G_gw || !G_gw_cas || !G_cc_cas || !G_out) {
        set_last_error("ccgf_self_energy_correction: sizes >= 1, nact <= nmo, non-NULL arrays required");
        return CCGF_ERR_INVALID_ARG;
    }
    const size_t smem = sizeof(double2) * ((size_t)nmo * nmo + (size_t)nact * nact * 2 + (size_t)nmo * nact + nmo) +
                        sizeof(int) * nmo + 16;
    if (smem > 220 * 1024) {
        set_last_error("ccgf_self_energy_correction: nmo too large for the per-(k, w) shared-memory inversion (nmo <= 110)");
        return CCGF_ERR_INVALID_ARG;
    }
    if ((i64)nk * nomega > 2147483647LL) {
        set_last_error("ccgf_self_energy_correction: nk * nomega too large");
        return CCGF_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    DBuf<int> err;
    CCGF_TRY(dalloc(err, 1));
    CCGF_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    CCGF_CUDA_TRY(cudaFuncSetAttribute(self_energy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    self_energy_kernel<<<(unsigned)((i64)nk * nomega), 256, smem, st>>>(nomega, nmo, nact, (const double2 *)V, (const double2 *)G_gw,
                                                                      (const double2 *)G_gw_cas, (const double2 *)G_cc_cas,
                                                                      (double2 *)G_out, err.p);
    CCGF_CUDA_TRY(cudaGetLastError());
    int flag = 0;
    CCGF_CUDA_TRY(cudaMemcpyAsync(&flag, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    if (flag) {
        set_last_error("ccgf_self_energy_correction: a matrix to invert is singular");
        return CCGF_ERR_INVALID_ARG;
    }
    return CCGF_OK;
}
