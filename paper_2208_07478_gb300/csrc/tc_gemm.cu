// Complex single-precision batched GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// C_b = alpha * sum_r A_{b,r} B_{b,r} + beta * C_b with float2 (interleaved complex) operands and the
// same descriptor as the SIMT kernels (GemmDesc). The complex product is a real GEMM through the
// embedding
//   A'[m][2k] = Re A[m][k], A'[m][2k+1] = Im A[m][k]             (A's own interleaved storage)
//   B'[2k][2n] = Re B, B'[2k+1][2n] = -Im B, B'[2k][2n+1] = Im B, B'[2k+1][2n+1] = Re B
//   C'[m][2n] = Re C, C'[m][2n+1] = Im C
// so one CTA computes a 128 x (2 BN) real tile = 128 x BN complex outputs in TMEM.
//
// Accuracy: every operand x is split into TF32 parts hi = rn_tf32(x), lo = rn_tf32(x - hi), and each
// K-step issues three tcgen05.mma.kind::tf32 (hi*hi + hi*lo + lo*hi) accumulating in FP32, which
// keeps the product near single-precision accuracy (the dropped lo*lo term is below 2^-22 relative).
//
// Shared memory holds each operand tile in the K-major, no-swizzle canonical layout of the MMA
// descriptors: 8-row x 16-byte core matrices, 128 bytes apart along K (leading byte offset) and
// 1024 bytes apart along M/N (stride byte offset). Two stages: the 256 threads stage tile s+1
// (global loads, TF32 split, conflict-free 16-byte shared stores) while the MMAs of tile s run; one
// thread issues the MMAs and commits them to the stage's mbarrier. Every wait is bounded: on timeout
// the CTA records an error flag, stops issuing, waits (bounded) for its committed MMAs, frees its
// TMEM and returns without writing C.
#include "ccgf_internal.h"
#include <cstdint>

namespace {

constexpr int BM = 128;          // rows per CTA = MMA M = TMEM lanes
constexpr int BKC = 16;          // complex K per stage (32 real K = one 128-byte core-matrix row strip)
constexpr int NTHREADS = 256;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s per wait (one tile of MMAs takes microseconds)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start >> 4, LBO = 128 B, SBO = 1024 B, fixed 0b001 at bit 46,
// base offset 0, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor for kind::tf32: D = F32 (bits 4-5), A = B = TF32 (bits 7-9, 10-12), both
// K-major (bits 15, 16 clear), N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t make_idesc(int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ float rn_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
__device__ __forceinline__ void split(float x, float &hi, float &lo) {
    hi = rn_tf32(x);
    lo = rn_tf32(x - hi);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait for the completion of the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity) {
    const uint32_t a = smem_u32(bar);
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned it = 0; it < (1u << 30); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255) == 255 && globaltimer_ns() - t0 > kWaitLimitNs) return false;
    }
    return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void st_shared4(unsigned char *p, float a, float b, float c, float d) {
    *(float4 *)p = make_float4(a, b, c, d);
}

template <int NCOLS>
__global__ void __launch_bounds__(NTHREADS, 1) tc_zgemm_kernel(GemmDesc d, const float2 *__restrict__ A, const float2 *__restrict__ B,
                                                               float2 *__restrict__ C, int BNc, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int NR = 2 * BNc;                                  // real rows of the B' tile (multiple of 16)
    const uint32_t a_bytes = BM * 2 * BKC * 4;               // 16 KB
    const uint32_t b_bytes = (uint32_t)NR * 2 * BKC * 4;     // NR * 128 B
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;  // A hi | A lo | B hi | B lo
    uint64_t *bars = (uint64_t *)(smem_raw + 2 * stage_bytes);
    uint32_t *tmem_slot = (uint32_t *)(bars + 2);
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.z;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BNc;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)), "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    const int ktiles = (d.K + BKC - 1) / BKC;
    const int total = d.nred * ktiles;
    const uint32_t idesc = make_idesc(NR);
    int issued = 0;

    for (int kt = 0; kt < total; ++kt) {
        const int st = kt & 1;
        if (kt >= 2 && !mbar_wait(&bars[st], ((kt - 2) >> 1) & 1)) {
            // the MMAs that read this stage two tiles ago did not finish in time
            atomicExch(err, 1);
            abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) break;
        const int r = kt / ktiles, k0 = (kt % ktiles) * BKC;
        const float2 *Ab = A + d.offA[(i64)b * d.nred + r];
        const float2 *Bb = B + d.offB[(i64)b * d.nred + r];
        unsigned char *sAh = smem_raw + st * stage_bytes, *sAl = sAh + a_bytes, *sBh = sAl + a_bytes, *sBl = sBh + b_bytes;

        // A: 32 warp tasks of 8 rows x 8 complex k; lane = (row r8, pair c) writes one 16-byte chunk
        // (2 complex k) of core matrix (group g, K index kh*4 + c) in the hi and lo tiles
        {
            const int r8 = lane & 7, c = lane >> 3;
            for (int t = warp; t < 32; t += NTHREADS / 32) {
                const int g = t >> 1, kh = t & 1;
                const int m = m0 + g * 8 + r8, k = k0 + kh * 8 + c * 2;
                float2 v0 = make_float2(0.f, 0.f), v1 = v0;
                if (m < d.M) {
                    const float2 *row = Ab + (i64)m * d.rsA;
                    if (k < d.K) v0 = row[(i64)k * d.csA];
                    if (k + 1 < d.K) v1 = row[(i64)(k + 1) * d.csA];
                }
                float h0, l0, h1, l1, h2, l2, h3, l3;
                split(v0.x, h0, l0);
                split(v0.y, h1, l1);
                split(v1.x, h2, l2);
                split(v1.y, h3, l3);
                const uint32_t off = g * 1024 + (kh * 4 + c) * 128 + r8 * 16;
                st_shared4(sAh + off, h0, h1, h2, h3);
                st_shared4(sAl + off, l0, l1, l2, l3);
            }
        }
        // B': BNc / 4 warp tasks of 4 complex n (8 real rows = one core-matrix group) x 16 complex k;
        // lane = (n nl, k pair kp) writes rows 2nl and 2nl+1 of core matrix kp, odd kp starting with
        // the second row so that the 8 lanes of each store phase hit distinct banks
        {
            const int nl = lane & 3, kp = lane >> 2;
            for (int t = warp; t < BNc / 4; t += NTHREADS / 32) {
                const int n = n0 + t * 4 + nl, k = k0 + kp * 2;
                float2 v0 = make_float2(0.f, 0.f), v1 = v0;
                if (n < d.N) {
                    const float2 *col = Bb + (i64)n * d.csB;
                    if (k < d.K) v0 = col[(i64)k * d.rsB];
                    if (k + 1 < d.K) v1 = col[(i64)(k + 1) * d.rsB];
                }
                float rh0, rl0, ih0, il0, rh1, rl1, ih1, il1;
                split(v0.x, rh0, rl0);
                split(v0.y, ih0, il0);
                split(v1.x, rh1, rl1);
                split(v1.y, ih1, il1);
                const uint32_t base = t * 1024 + kp * 128 + (2 * nl) * 16;
                const uint32_t o_re = base, o_im = base + 16;   // row 2n: (Re, -Im), row 2n+1: (Im, Re)
                if (kp & 1) {
                    st_shared4(sBh + o_im, ih0, rh0, ih1, rh1);
                    st_shared4(sBh + o_re, rh0, -ih0, rh1, -ih1);
                    st_shared4(sBl + o_im, il0, rl0, il1, rl1);
                    st_shared4(sBl + o_re, rl0, -il0, rl1, -il1);
                } else {
                    st_shared4(sBh + o_re, rh0, -ih0, rh1, -ih1);
                    st_shared4(sBh + o_im, ih0, rh0, ih1, rh1);
                    st_shared4(sBl + o_re, rl0, -il0, rl1, -il1);
                    st_shared4(sBl + o_im, il0, rl0, il1, rl1);
                }
            }
        }
        // generic-proxy shared stores -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t aH = smem_u32(sAh), aL = smem_u32(sAl), bH = smem_u32(sBh), bL = smem_u32(sBl);
#pragma unroll
            for (int ks = 0; ks < (2 * BKC) / 8; ++ks) {   // 8 real K per MMA = two core matrices = 256 B
                const uint32_t off = ks * 256;
                const uint64_t dah = make_desc(aH + off), dal = make_desc(aL + off);
                const uint64_t dbh = make_desc(bH + off), dbl = make_desc(bL + off);
                mma_tf32(tmem, dah, dbh, idesc, (kt > 0 || ks > 0) ? 1u : 0u);
                mma_tf32(tmem, dah, dbl, idesc, 1u);
                mma_tf32(tmem, dal, dbh, idesc, 1u);
            }
            // arrives on the stage barrier once every MMA issued so far by this thread has completed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&bars[st]))
                         : "memory");
        }
        issued = kt + 1;
    }
    if (issued > 0) {
        const int last = issued - 1;
        if (!mbar_wait(&bars[last & 1], (last >> 1) & 1)) {
            atomicExch(err, 1);
            abort_flag = 1;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_flag && issued > 0) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (one output row per thread) and every
        // other 8-column chunk starting at chunk w / 4; alpha, beta applied in FP32
        const int quarter = warp & 3, half = warp >> 2;
        const int m = m0 + quarter * 32 + lane;
        const float ax = (float)d.alpha.x, ay = (float)d.alpha.y, bx = (float)d.beta.x, by = (float)d.beta.y;
        const bool use_beta = (d.beta.x != 0.0 || d.beta.y != 0.0);
        float2 *Cb = C + d.offC[b];
        for (int c0 = half * 8; c0 < NR; c0 += 16) {
            uint32_t v[8];
            const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m < d.M) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int n = n0 + (c0 >> 1) + q;
                    if (n >= d.N) continue;
                    const float re = __uint_as_float(v[2 * q]), im = __uint_as_float(v[2 * q + 1]);
                    float2 *cp = Cb + (i64)m * d.rsC + (i64)n * d.csC;
                    float2 o;
                    o.x = ax * re - ay * im;
                    o.y = ax * im + ay * re;
                    if (use_beta) {
                        const float2 cv = *cp;
                        o.x += bx * cv.x - by * cv.y;
                        o.y += bx * cv.y + by * cv.x;
                    }
                    *cp = o;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
}

template <int NCOLS>
void launch_cols(dim3 grid, size_t smem, cudaStream_t st, const GemmDesc &d, const float2 *A, const float2 *B, float2 *C, int BNc,
                 int *err) {
    cudaFuncSetAttribute(tc_zgemm_kernel<NCOLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc_zgemm_kernel<NCOLS><<<grid, NTHREADS, smem, st>>>(d, A, B, C, BNc, err);
}

}  // namespace

bool tc_zgemm_supported(const GemmDesc &d) {
    // worth a 128-row tile, and within the grid limits of one launch
    return d.M >= 32 && d.N >= 8 && d.K >= 8 && d.nred >= 1 && d.batch >= 1 && d.batch <= 65535 && ceil_div(d.M, BM) <= 65535;
}

size_t tc_zgemm_smem_bytes(int BNc) {
    const size_t stage = (size_t)2 * BM * 2 * BKC * 4 + (size_t)2 * (2 * BNc) * 2 * BKC * 4;
    return 2 * stage + 64;
}

int launch_tc_zgemm(const GemmDesc &d, const float2 *A, const float2 *B, float2 *C, int *err, cudaStream_t st) {
    // complex N tile: 128 (256 real TMEM columns), or N rounded up to a multiple of 8 when smaller
    const int BNc = d.N >= 128 ? 128 : (int)ceil_div(d.N, 8) * 8;
    const int NR = 2 * BNc;
    const size_t smem = tc_zgemm_smem_bytes(BNc);
    const dim3 grid((unsigned)ceil_div(d.N, BNc), (unsigned)ceil_div(d.M, BM), (unsigned)d.batch);
    if (NR <= 32)
        launch_cols<32>(grid, smem, st, d, A, B, C, BNc, err);
    else if (NR <= 64)
        launch_cols<64>(grid, smem, st, d, A, B, C, BNc, err);
    else if (NR <= 128)
        launch_cols<128>(grid, smem, st, d, A, B, C, BNc, err);
    else
        launch_cols<256>(grid, smem, st, d, A, B, C, BNc, err);
    return 1;
}
