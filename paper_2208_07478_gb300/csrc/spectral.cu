// Spectral function and density of states (Eq. 10): A(k, w) = -(1/pi) Im G(k, w), whose trace over
// the orbitals is the k-resolved density of states.
//
// ccgf_solve_gf returns the time-ordered G of Eq. 9 (G+ with +i eta, G- with -i eta). Its removal part
// then has Im G- > 0 at its poles, so -(1/pi) Im Tr G is negative below the gap. With the two parts
// given separately the removal part enters with the opposite sign (the retarded convention), which
// gives positive peaks on both sides: dos = -(1/pi) Im Tr G+ + (1/pi) Im Tr G-.
#include "ccgf_internal.h"
#include <cmath>

namespace {

// one thread block per (k, w): dos[k][w] = sign_p * (-(1/pi)) Im sum_p G[k][w][p][p] (+ the removal part)
__global__ void dos_kernel(int nomega, int nmo, const double2 *__restrict__ G, const double2 *__restrict__ Gm, double *dos) {
    const i64 kw = blockIdx.x;
    const double2 *g = G + kw * (i64)nmo * nmo;
    const double2 *gm = Gm ? Gm + kw * (i64)nmo * nmo : nullptr;
    double acc = 0.0;
    for (int p = threadIdx.x; p < nmo; p += blockDim.x) {
        acc -= g[(i64)p * nmo + p].y;
        if (gm) acc += gm[(i64)p * nmo + p].y;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) dos[kw] = red[0] / M_PI;
    (void)nomega;
}

// dos_total[w] = (1/nk) sum_k dos[k][w]
__global__ void dos_total_kernel(int nk, int nomega, const double *__restrict__ dos, double *total) {
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nomega; w += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < nk; ++k) acc += dos[(i64)k * nomega + w];
        total[w] = acc / nk;
    }
}

}  // namespace

extern "C" ccgf_status ccgf_spectral_function(int nk, int nomega, int nmo, const double *G, const double *G_minus, double *dos,
                                              double *dos_total, void *stream) {
    if (nk < 1 || nomega < 1 || nmo < 1 || !G || !dos) {
        set_last_error("ccgf_spectral_function: nk, nomega, nmo >= 1 and non-NULL G, dos required");
        return CCGF_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const i64 nkw = (i64)nk * nomega;
    if (nkw > 2147483647LL) {
        set_last_error("ccgf_spectral_function: nk * nomega too large");
        return CCGF_ERR_INVALID_ARG;
    }
    dos_kernel<<<(unsigned)nkw, 256, 0, st>>>(nomega, nmo, (const double2 *)G, (const double2 *)G_minus, dos);
    if (dos_total) dos_total_kernel<<<(unsigned)ceil_div(nomega, 256), 256, 0, st>>>(nk, nomega, dos, dos_total);
    CCGF_CUDA_TRY(cudaGetLastError());
    return CCGF_OK;
}
