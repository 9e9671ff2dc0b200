// ccgf_sigma_ip_noalloc: the EOM-IP sigma of ccgf_sigma_ip (FP64) for callers that
// must not allocate device memory during a call.
//
// Some callers cannot call cudaMalloc at the point where they need a sigma product:
// a host framework that owns all device memory through its own pool and forbids
// foreign allocations, a latency-critical loop where the device-wide synchronisation
// that cudaMalloc / cudaFree may imply is not acceptable, or a process that has
// already reserved the whole device memory for other buffers. For them this entry
// point runs the same plan of GEMM and permute kernels as ccgf_sigma_ip, with every
// scratch buffer it needs (the layout transposes of the input and the output, the
// plan's offset table, the GEMM and permute temporaries and the split-K partial
// sums) placed in one file-scope static device array of fixed size. The caller
// still passes the handle (built earlier), the input vectors and the output vectors.
//
// Properties callers rely on:
//   - Size limit: CCGF_NOALLOC_SCRATCH_BYTES (32 MiB) per device, held by every GPU
//     that loads the library until the process exits. The first 1 MiB holds the
//     offset table (131072 entries), the rest the complex scratch (1,966,080
//     elements). A call whose (dimension, nvec) needs more returns
//     CCGF_ERR_INVALID_ARG and says how much it would need.
//   - The first call on each device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it.
//   - All calls share the one array and leave their contents in it. Every scratch
//     element is written before it is read within a call, so nothing has to start
//     at zero; but calls whose kernels overlap on the GPU (different streams, or
//     different host threads without ordering) race on the array: order them.
//   - No cudaMalloc, cudaFree or allocating library routine is called.
#include "ccgf_internal.h"
#include <mutex>

#define CCGF_NOALLOC_SCRATCH_BYTES (32u << 20)
#define CCGF_NOALLOC_OFFSET_BYTES (1u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[CCGF_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device (the host-side name of
// the array is only a stand-in and must never be handed to a kernel).
ccgf_status scratch_address(void **out) {
    int dev = 0;
    CCGF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_last_error("device index beyond the supported range");
        return CCGF_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            set_last_error(std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
            return CCGF_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return CCGF_OK;
}

}  // namespace

extern "C" ccgf_status ccgf_sigma_ip_noalloc(ccgf_handle *h, int kshift, long long nvec, const double *x, double *y,
                                             void *stream) {
    if (!h || !x || !y) { set_last_error("NULL handle or vector"); return CCGF_ERR_INVALID_ARG; }
    if (kshift < 0 || kshift >= h->nk) { set_last_error("kshift out of range"); return CCGF_ERR_INVALID_ARG; }
    if (nvec < 1 || nvec > 65536) { set_last_error("nvec must be in [1, 65536]"); return CCGF_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const i64 D = h->dim_ip;
    const int nv = (int)nvec;
    const i64 cap = (CCGF_NOALLOC_SCRATCH_BYTES - CCGF_NOALLOC_OFFSET_BYTES) / sizeof(double2);
    // input transpose + output transpose + the plan's own arena
    const i64 need = 2 * D * nv + sigma_arena_elems(h, nv);
    if (need > cap) {
        set_last_error("ccgf_sigma_ip_noalloc: nvec " + std::to_string(nvec) + " needs " + std::to_string(need) +
                       " complex scratch elements, the static workspace holds " + std::to_string(cap));
        return CCGF_ERR_INVALID_ARG;
    }
    void *base = nullptr;
    CCGF_TRY(scratch_address(&base));
    i64 *offsets = (i64 *)base;
    double2 *cplx = (double2 *)((unsigned char *)base + CCGF_NOALLOC_OFFSET_BYTES);
    double2 *xt = cplx, *yt = cplx + D * nv, *arena = cplx + 2 * D * nv;
    launch_transpose_in((const double2 *)x, xt, D, nv, nv, st);
    ccgf_status s = sigma_apply_in_arena(h, CCGF_SECTOR_IP, kshift, nv, xt, yt, arena, cap - 2 * D * nv, offsets,
                                         CCGF_NOALLOC_OFFSET_BYTES / sizeof(i64), st);
    if (s != CCGF_OK) return s;
    launch_transpose_out(yt, (double2 *)y, D, nv, nv, st);
    h->launches += 2;
    CCGF_CUDA_TRY(cudaGetLastError());
    return CCGF_OK;
}
