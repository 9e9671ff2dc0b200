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
// Three kernels share this arithmetic and differ in how operands reach shared memory:
//  - tc_zgemm_kernel (register-fed, any A): 256 threads load both tiles, split them and store them
//    in the K-major no-swizzle canonical layout (8-row x 16-byte core matrices, 128 B apart along K,
//    1024 B apart along M/N), two stages; one thread issues the MMAs.
//  - tc_zgemm_tma_kernel: A by TMA (128-byte swizzle) from TF32 hi / lo copies of the intermediate,
//    B' staged by four producer warps, up to four stages.
//  - tc_zgemm_bulk_kernel: A by TMA (64-byte swizzle) and B' by one cp.async.bulk per stage from an
//    image expanded just before by bimage_kernel; no thread stages data, up to eight stages.
// Every wait is bounded: on timeout the CTA records an error flag, stops issuing, waits (bounded)
// for its issued copies and MMAs, frees its TMEM and returns without writing C.
#include "ccgf_internal.h"
#include <cuda.h>
#include <atomic>
#include <cstdio>
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

namespace {

constexpr int BM = 128;          // rows per CTA = MMA M = TMEM lanes
constexpr int BKC = 16;          // complex K per stage (32 real K = one 128-byte core-matrix row strip)
constexpr int NTHREADS = 256;
// Every wait is bounded by GemmDesc::wait_ns (the handle's device_wait_timeout_ms; one tile of MMAs
// takes microseconds); kWaitLimitNs applies where a kernel has no descriptor.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

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
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned long long limit_ns = kWaitLimitNs) {
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
        if ((it & 255) == 255 && globaltimer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// descriptor copy with the wait bound set (0 = the default bound)
inline GemmDesc with_wait_limit(const GemmDesc &d) {
    GemmDesc o = d;
    if (o.wait_ns == 0) o.wait_ns = kWaitLimitNs;
    return o;
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

__device__ __forceinline__ float2 as_f2(float2 a) { return a; }
__device__ __forceinline__ float2 as_f2(double2 a) { return make_float2((float)a.x, (float)a.y); }

// TA: storage type of A (double2: an FP64 intermediate without an FP32 copy, rounded as it is loaded)
template <int NCOLS, typename TA = float2>
__global__ void __launch_bounds__(NTHREADS, 1) tc_zgemm_kernel(GemmDesc d, const TA *__restrict__ A, const float2 *__restrict__ B,
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

    // The operands of stage kt + 1 are loaded into registers (A rounded to FP32 on load) right after
    // stage kt is split into shared memory, so their global-load latency overlaps the tensor cores'
    // work on stage kt instead of following it. 32 A tasks (8 rows x 8 complex k) and at most 32 B
    // tasks (4 complex n x 16 complex k): four of each per warp.
    float2 ra[4][2], rb[4][2];
    auto load_regs = [&](int kt) {
        const int r = kt / ktiles, k0 = (kt % ktiles) * BKC;
        const TA *Ab = A + d.offA[(i64)b * d.nred + r];
        const float2 *Bb = B + d.offB[(i64)b * d.nred + r];
        const int r8 = lane & 7, c = lane >> 3, nl = lane & 3, kp = lane >> 2;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = warp + q * (NTHREADS / 32);
            const int g = t >> 1, kh = t & 1;
            const int m = m0 + g * 8 + r8, k = k0 + kh * 8 + c * 2;
            float2 v0 = make_float2(0.f, 0.f), v1 = v0;
            if (m < d.M) {
                const TA *row = Ab + (i64)m * d.rsA;
                if (k < d.K) v0 = as_f2(row[(i64)k * d.csA]);
                if (k + 1 < d.K) v1 = as_f2(row[(i64)(k + 1) * d.csA]);
            }
            ra[q][0] = v0;
            ra[q][1] = v1;
            float2 u0 = make_float2(0.f, 0.f), u1 = u0;
            const int n = n0 + t * 4 + nl, kb = k0 + kp * 2;
            if (t < BNc / 4 && n < d.N) {
                const float2 *col = Bb + (i64)n * d.csB;
                if (kb < d.K) u0 = col[(i64)kb * d.rsB];
                if (kb + 1 < d.K) u1 = col[(i64)(kb + 1) * d.rsB];
            }
            rb[q][0] = u0;
            rb[q][1] = u1;
        }
    };
    if (total > 0) load_regs(0);

    for (int kt = 0; kt < total; ++kt) {
        const int st = kt & 1;
        if (kt >= 2 && !mbar_wait(&bars[st], ((kt - 2) >> 1) & 1, d.wait_ns)) {
            // the MMAs that read this stage two tiles ago did not finish in time
            atomicExch(err, 1);
            abort_flag = 1;
        }
        __syncthreads();
        if (abort_flag) break;
        unsigned char *sAh = smem_raw + st * stage_bytes, *sAl = sAh + a_bytes, *sBh = sAl + a_bytes, *sBl = sBh + b_bytes;
        {
            // A: lane = (row r8, pair c) writes one 16-byte chunk (2 complex k) of core matrix (group g,
            // K index kh*4 + c) in the hi and lo tiles
            const int r8 = lane & 7, c = lane >> 3;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int t = warp + q * (NTHREADS / 32);
                const int g = t >> 1, kh = t & 1;
                float h0, l0, h1, l1, h2, l2, h3, l3;
                split(ra[q][0].x, h0, l0);
                split(ra[q][0].y, h1, l1);
                split(ra[q][1].x, h2, l2);
                split(ra[q][1].y, h3, l3);
                const uint32_t off = g * 1024 + (kh * 4 + c) * 128 + r8 * 16;
                st_shared4(sAh + off, h0, h1, h2, h3);
                st_shared4(sAl + off, l0, l1, l2, l3);
            }
        }
        {
            // B': lane = (n nl, k pair kp) writes rows 2nl and 2nl+1 of core matrix kp, odd kp starting
            // with the second row so that the 8 lanes of each store phase hit distinct banks
            const int nl = lane & 3, kp = lane >> 2;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int t = warp + q * (NTHREADS / 32);
                if (t >= BNc / 4) continue;
                float rh0, rl0, ih0, il0, rh1, rl1, ih1, il1;
                split(rb[q][0].x, rh0, rl0);
                split(rb[q][0].y, ih0, il0);
                split(rb[q][1].x, rh1, rl1);
                split(rb[q][1].y, ih1, il1);
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
        if (kt + 1 < total) load_regs(kt + 1);
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
        if (!mbar_wait(&bars[last & 1], (last >> 1) & 1, d.wait_ns)) {
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

template <int NCOLS, typename TA>
void launch_cols(dim3 grid, size_t smem, cudaStream_t st, const GemmDesc &d, const TA *A, const float2 *B, float2 *C, int BNc,
                 int *err) {
    cudaFuncSetAttribute(tc_zgemm_kernel<NCOLS, TA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc_zgemm_kernel<NCOLS, TA><<<grid, NTHREADS, smem, st>>>(with_wait_limit(d), A, B, C, BNc, err);
}


// ----------------------------------------------------------------------------- TMA-fed variant
// The A operand (an intermediate: fixed for the handle's lifetime) is pre-split once into TF32
// hi / lo copies with A's own layout; TMA loads 128-row x 32-float boxes of both into shared memory
// with the 128-byte swizzle (the canonical SW128 K-major layout of the MMA descriptor). Roles:
//   warps 0-3  stage B' hi / lo from registers (as above), then run the epilogue (TMEM lane quarter = warp)
//   warp 4     lane 0 issues the TMA loads of A
//   warp 5     allocates TMEM; lane 0 issues the MMAs and commits them
// Barriers per stage: fullA (TMA bytes), fullB (4 warp arrivals), empty (MMA commit); one more
// barrier signals the finished accumulator to the epilogue.
constexpr int TMA_THREADS = 192;
constexpr int MAX_STAGES = 4;

__device__ __forceinline__ uint64_t make_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset: unused for swizzled K-major
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;             // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// bounded wait that also gives up as soon as another role has aborted the CTA
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, unsigned parity, volatile int *abort_flag,
                                                   unsigned long long limit_ns) {
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
        if ((it & 255) == 255 && (*abort_flag || globaltimer_ns() - t0 > limit_ns)) return false;
    }
    return false;
}

template <int NCOLS>
__global__ void __launch_bounds__(TMA_THREADS, 1)
    tc_zgemm_tma_kernel(GemmDesc d, const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
                        const i64 *__restrict__ rowA, const float2 *__restrict__ B, float2 *__restrict__ C, int BNc, int S,
                        int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned base (the 128-byte swizzle pattern repeats every 8 rows = 1024 B)
    unsigned char *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const int NR = 2 * BNc;
    const uint32_t a_bytes = BM * 2 * BKC * 4;   // 16 KB per part
    const uint32_t b_bytes = (uint32_t)NR * 2 * BKC * 4;
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    uint64_t *fullA = (uint64_t *)(base + S * stage_bytes);
    uint64_t *fullB = fullA + MAX_STAGES;
    uint64_t *empty = fullB + MAX_STAGES;
    uint64_t *accum = empty + MAX_STAGES;
    uint32_t *tmem_slot = (uint32_t *)(accum + 1);
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.z;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BNc;
    const int ktiles = (d.K + BKC - 1) / BKC;
    const int total = d.nred * ktiles;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&fullA[s], 1);
            mbar_init(&fullB[s], 4);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)), "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    volatile int *abort_v = &abort_flag;

    if (warp == 4) {
        if (lane == 0) {
            // A producer
            int issued = 0;
            for (int kt = 0; kt < total; ++kt) {
                const int s = kt % S;
                if (kt >= S && !mbar_wait_or_abort(&empty[s], ((kt / S) - 1) & 1, abort_v, d.wait_ns)) {
                    atomicExch(err, 1);
                    *abort_v = 1;
                    break;
                }
                const int r = kt / ktiles, k0 = (kt % ktiles) * BKC;
                const int y = (int)rowA[(i64)b * d.nred + r] + m0;
                unsigned char *sA = base + s * stage_bytes;
                mbar_expect_tx(&fullA[s], 2 * a_bytes);
                tma_load_2d(smem_u32(sA), &map_hi, 2 * k0, y, &fullA[s]);
                tma_load_2d(smem_u32(sA + a_bytes), &map_lo, 2 * k0, y, &fullA[s]);
                issued = kt + 1;
            }
            // no copy may still be writing shared memory when the CTA exits
            for (int kt = issued - S > 0 ? issued - S : 0; kt < issued; ++kt)
                if (!mbar_wait(&fullA[kt % S], (kt / S) & 1, d.wait_ns)) atomicExch(err, 1);
        }
    } else if (warp == 5) {
        if (lane == 0) {
            // MMA issuer
            const uint32_t idesc = make_idesc(NR);
            int issued = 0;
            for (int kt = 0; kt < total; ++kt) {
                const int s = kt % S;
                const unsigned par = (kt / S) & 1;
                if (!mbar_wait_or_abort(&fullA[s], par, abort_v, d.wait_ns) || !mbar_wait_or_abort(&fullB[s], par, abort_v, d.wait_ns)) {
                    atomicExch(err, 1);
                    *abort_v = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                unsigned char *sA = base + s * stage_bytes;
                const uint32_t aH = smem_u32(sA), aL = aH + a_bytes, bH = aL + a_bytes, bL = bH + b_bytes;
#pragma unroll
                for (int ks = 0; ks < (2 * BKC) / 8; ++ks) {
                    const uint64_t dah = make_desc_sw128(aH + ks * 32), dal = make_desc_sw128(aL + ks * 32);
                    const uint64_t dbh = make_desc(bH + ks * 256), dbl = make_desc(bL + ks * 256);
                    mma_tf32(tmem, dah, dbh, idesc, (kt > 0 || ks > 0) ? 1u : 0u);
                    mma_tf32(tmem, dah, dbl, idesc, 1u);
                    mma_tf32(tmem, dal, dbh, idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&empty[s]))
                             : "memory");
                issued = kt + 1;
            }
            // the accumulator barrier fires when every MMA issued above has completed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(accum))
                         : "memory");
            if (issued < total) *abort_v = 1;
        }
    } else {
        // B' producers (warps 0-3), then the epilogue
        const int nl = lane & 3, kp = lane >> 2;
        for (int kt = 0; kt < total; ++kt) {
            const int s = kt % S;
            if (kt >= S && !mbar_wait_or_abort(&empty[s], ((kt / S) - 1) & 1, abort_v, d.wait_ns)) {
                atomicExch(err, 1);
                *abort_v = 1;
                break;
            }
            const int r = kt / ktiles, k0 = (kt % ktiles) * BKC;
            const float2 *Bb = B + d.offB[(i64)b * d.nred + r];
            unsigned char *sBh = base + s * stage_bytes + 2 * a_bytes, *sBl = sBh + b_bytes;
            const int k = k0 + kp * 2;
            for (int t0 = warp; t0 < BNc / 4; t0 += 32) {
                // up to 8 tasks per warp: all loads first, then the split and the stores
                float2 v0[8], v1[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int t = t0 + 4 * q;
                    v0[q] = make_float2(0.f, 0.f);
                    v1[q] = v0[q];
                    const int n = n0 + t * 4 + nl;
                    if (t < BNc / 4 && n < d.N) {
                        const float2 *col = Bb + (i64)n * d.csB;
                        if (k < d.K) v0[q] = col[(i64)k * d.rsB];
                        if (k + 1 < d.K) v1[q] = col[(i64)(k + 1) * d.rsB];
                    }
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int t = t0 + 4 * q;
                    if (t >= BNc / 4) break;
                    float rh0, rl0, ih0, il0, rh1, rl1, ih1, il1;
                    split(v0[q].x, rh0, rl0);
                    split(v0[q].y, ih0, il0);
                    split(v1[q].x, rh1, rl1);
                    split(v1[q].y, ih1, il1);
                    const uint32_t o_re = t * 1024 + kp * 128 + (2 * nl) * 16, o_im = o_re + 16;
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
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&fullB[s]);
        }
        // epilogue: wait for the accumulator, then TMEM -> registers -> C
        const bool ok = mbar_wait_or_abort(accum, 0, abort_v, d.wait_ns);
        if (!ok) atomicExch(err, 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (__all_sync(0xffffffffu, ok && !*abort_v)) {
            const int m = m0 + warp * 32 + lane;
            const float ax = (float)d.alpha.x, ay = (float)d.alpha.y, bx = (float)d.beta.x, by = (float)d.beta.y;
            const bool use_beta = (d.beta.x != 0.0 || d.beta.y != 0.0);
            float2 *Cb = C + d.offC[b];
            for (int c0 = 0; c0 < NR; c0 += 8) {
                uint32_t v[8];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
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
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 5) {
        // every MMA this CTA issued has completed once the accumulator barrier fired; after an
        // abort, wait for it (bounded) before the columns are released
        if (*abort_v) {
            if (!mbar_wait(accum, 0, d.wait_ns)) atomicExch(err, 1);
            __syncwarp();
        }
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
    }
}

__global__ void tf32_split_kernel(const float2 *__restrict__ a, float2 *__restrict__ hi, float2 *__restrict__ lo, i64 n) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
        const float2 v = a[i];
        float hx, lx, hy, ly;
        split(v.x, hx, lx);
        split(v.y, hy, ly);
        hi[i] = make_float2(hx, hy);
        lo[i] = make_float2(lx, ly);
    }
}

template <int NCOLS>
void launch_tma_cols(dim3 grid, size_t smem, cudaStream_t st, const GemmDesc &d, const CUtensorMap &mh, const CUtensorMap &ml,
                     const i64 *rowA, const float2 *B, float2 *C, int BNc, int S, int *err) {
    cudaFuncSetAttribute(tc_zgemm_tma_kernel<NCOLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc_zgemm_tma_kernel<NCOLS><<<grid, TMA_THREADS, smem, st>>>(with_wait_limit(d), mh, ml, rowA, B, C, BNc, S, err);
}


// ----------------------------------------------------------------------------- bulk-fed variant
// Both operands arrive by asynchronous copies, so no thread stages data in the main loop:
//  - A by TMA (64-byte swizzle, 128 rows x 16 floats = 8 complex K per stage) from the TF32
//    hi / lo copies;
//  - B' from an image written just before by bimage_kernel: for every distinct B block (slot),
//    N tile and K tile, the TF32 hi then lo parts of the 2x2-embedded tile in the canonical
//    no-swizzle K-major layout (8-row groups 512 B apart, core matrices 128 B apart along K),
//    fetched with one cp.async.bulk per stage.
// Warp 0 lane 0 produces, warp 1 allocates TMEM and its lane 0 issues the MMAs, warps 2-5 run
// the epilogue (TMEM lane quarter = warp % 4). Up to 8 stages of 16 real K each.
constexpr int BKC3 = 8;                  // complex K per stage
constexpr int MAX_STAGES3 = 8;

// complex N tile of the bulk-fed kernel: N rounded up to 8 when it fits one tile; otherwise the
// width in 64..128 (multiples of 8) with the least modelled time: padded work, divided by the wave
// efficiency of one CTA per SM, times the shared-memory pressure of the tile (per MMA clock the
// operand reads take 8192 / NR + 64 bytes and the copies landing in shared memory 5461 / NR + 43,
// NR = 2 BN real columns, against 128 B/clk)
static int tc3_bn(const GemmDesc &d) {
    if (d.N <= 128) return (int)ceil_div(d.N, 8) * 8;
    const double mt = (double)ceil_div(d.M, BM) * d.batch;
    int best = 128;
    double best_cost = 1e300;
    for (int bn = 128; bn >= 64; bn -= 8) {
        const double nt = (double)ceil_div(d.N, bn);
        const double waves = nt * mt / 152.0;
        const double eff = waves >= 1.0 ? waves / std::ceil(waves) : waves;
        const double nr = 2.0 * bn;
        const double smem = std::max(1.0, (8192.0 / nr + 64.0 + 5461.0 / nr + 42.7) / 128.0);
        const double cost = nt * bn / eff * smem;
        if (cost < best_cost * (1 - 1e-9)) {
            best_cost = cost;
            best = bn;
        }
    }
    return best;
}

__device__ __forceinline__ uint64_t make_desc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset: unused for swizzled K-major
    d |= (uint64_t)(512 >> 4) << 32;    // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;             // 64-byte swizzle
    return d;
}
__device__ __forceinline__ uint64_t make_desc_k16(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;    // next core matrix along K
    d |= (uint64_t)(512 >> 4) << 32;    // next 8-row group
    d |= (uint64_t)1 << 46;
    return d;
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"((uint64_t)src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// B' image of the slots: thread = (slot, N tile, K tile, 4-column group t, k pair kp, column nl);
// writes rows 2n and 2n+1 (16 bytes each) of the hi part and of the lo part
__global__ void bimage_kernel(GemmDesc d, const float2 *__restrict__ B, const i64 *__restrict__ bsrc, int nslots, int BNc,
                              int ntiles, int ktiles, float *__restrict__ img) {
    const int NR = 2 * BNc;
    const i64 chunk = (i64)NR * 2 * (2 * BKC3);   // floats per (slot, N tile, K tile): hi + lo
    const i64 per_tile = (i64)(BNc / 4) * 16;       // threads per (slot, N tile, K tile)
    const i64 total = (i64)nslots * ntiles * ktiles * per_tile;
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (i64)gridDim.x * blockDim.x) {
        const int nl = (int)(i & 3), kp = (int)((i >> 2) & 3);
        i64 r = i >> 4;
        const int t = (int)(r % (BNc / 4));
        r /= (BNc / 4);
        const int kt = (int)(r % ktiles);
        r /= ktiles;
        const int nt = (int)(r % ntiles);
        const int slot = (int)(r / ntiles);
        const int n = nt * BNc + t * 4 + nl, k = kt * BKC3 + kp * 2;
        float2 v0 = make_float2(0.f, 0.f), v1 = v0;
        if (n < d.N) {
            const float2 *col = B + bsrc[slot] + (i64)n * d.csB;
            if (k < d.K) v0 = col[(i64)k * d.rsB];
            if (k + 1 < d.K) v1 = col[(i64)(k + 1) * d.rsB];
        }
        float rh0, rl0, ih0, il0, rh1, rl1, ih1, il1;
        split(v0.x, rh0, rl0);
        split(v0.y, ih0, il0);
        split(v1.x, rh1, rl1);
        split(v1.y, ih1, il1);
        float *hi = img + (((i64)slot * ntiles + nt) * ktiles + kt) * chunk;
        float *lo = hi + (i64)NR * (2 * BKC3);
        const int o_re = t * 128 + kp * 32 + nl * 8, o_im = o_re + 4;   // in floats: row 2n, row 2n+1
        *(float4 *)(hi + o_re) = make_float4(rh0, -ih0, rh1, -ih1);
        *(float4 *)(hi + o_im) = make_float4(ih0, rh0, ih1, rh1);
        *(float4 *)(lo + o_re) = make_float4(rl0, -il0, rl1, -il1);
        *(float4 *)(lo + o_im) = make_float4(il0, rl0, il1, rl1);
    }
}

template <int NCOLS>
__global__ void __launch_bounds__(TMA_THREADS, 1)
    tc_zgemm_bulk_kernel(GemmDesc d, const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
                         const i64 *__restrict__ rowA, const i64 *__restrict__ bslot, const float *__restrict__ img,
                         float2 *__restrict__ C, int BNc, int S, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    const int NR = 2 * BNc;
    const uint32_t a_bytes = BM * 2 * BKC3 * 4;                  // 8 KB per part
    const uint32_t b_bytes = (uint32_t)NR * 2 * (2 * BKC3) * 4;  // hi + lo
    const uint32_t stage_bytes = 2 * a_bytes + b_bytes;
    uint64_t *full = (uint64_t *)(base + S * stage_bytes);
    uint64_t *empty = full + MAX_STAGES3;
    uint64_t *accum = empty + MAX_STAGES3;
    uint32_t *tmem_slot = (uint32_t *)(accum + 1);
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.z, nt = blockIdx.x;
    const int m0 = blockIdx.y * BM, n0 = nt * BNc;
    const int ktiles = (d.K + BKC3 - 1) / BKC3;
    const int ntiles = gridDim.x;
    const int total = d.nred * ktiles;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)), "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    volatile int *abort_v = &abort_flag;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kt = 0; kt < total; ++kt) {
                const int s = kt % S;
                if (kt >= S && !mbar_wait_or_abort(&empty[s], ((kt / S) - 1) & 1, abort_v, d.wait_ns)) {
                    atomicExch(err, 1);
                    *abort_v = 1;
                    break;
                }
                const int r = kt / ktiles, kk = kt % ktiles;
                const i64 br = (i64)b * d.nred + r;
                const int y = (int)rowA[br] + m0;
                unsigned char *sA = base + s * stage_bytes;
                const float *src = img + (((i64)bslot[br] * ntiles + nt) * ktiles + kk) * ((i64)b_bytes / 4);
                mbar_expect_tx(&full[s], 2 * a_bytes + b_bytes);
                tma_load_2d(smem_u32(sA), &map_hi, 2 * kk * BKC3, y, &full[s]);
                tma_load_2d(smem_u32(sA + a_bytes), &map_lo, 2 * kk * BKC3, y, &full[s]);
                bulk_load(smem_u32(sA + 2 * a_bytes), src, b_bytes, &full[s]);
                issued = kt + 1;
            }
            for (int kt = issued - S > 0 ? issued - S : 0; kt < issued; ++kt)
                if (!mbar_wait(&full[kt % S], (kt / S) & 1, d.wait_ns)) atomicExch(err, 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = make_idesc(NR);
            int issued = 0;
            for (int kt = 0; kt < total; ++kt) {
                const int s = kt % S;
                if (!mbar_wait_or_abort(&full[s], (kt / S) & 1, abort_v, d.wait_ns)) {
                    atomicExch(err, 1);
                    *abort_v = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t aH = smem_u32(base + s * stage_bytes), aL = aH + a_bytes, bH = aL + a_bytes, bL = bH + b_bytes / 2;
#pragma unroll
                for (int ks = 0; ks < (2 * BKC3) / 8; ++ks) {
                    const uint64_t dah = make_desc_sw64(aH + ks * 32), dal = make_desc_sw64(aL + ks * 32);
                    const uint64_t dbh = make_desc_k16(bH + ks * 256), dbl = make_desc_k16(bL + ks * 256);
                    mma_tf32(tmem, dah, dbh, idesc, (kt > 0 || ks > 0) ? 1u : 0u);
                    mma_tf32(tmem, dah, dbl, idesc, 1u);
                    mma_tf32(tmem, dal, dbh, idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&empty[s]))
                             : "memory");
                issued = kt + 1;
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(accum))
                         : "memory");
            if (issued < total) *abort_v = 1;
        }
    } else {
        const int quarter = warp & 3;
        const bool ok = mbar_wait_or_abort(accum, 0, abort_v, d.wait_ns);
        if (!ok) atomicExch(err, 1);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (__all_sync(0xffffffffu, ok && !*abort_v)) {
            const int m = m0 + quarter * 32 + lane;
            const float ax = (float)d.alpha.x, ay = (float)d.alpha.y, bx = (float)d.beta.x, by = (float)d.beta.y;
            const bool use_beta = (d.beta.x != 0.0 || d.beta.y != 0.0);
            float2 *Cb = C + d.offC[b];
            for (int c0 = 0; c0 < NR; c0 += 8) {
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
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        if (*abort_v) {
            if (!mbar_wait(accum, 0, d.wait_ns)) atomicExch(err, 1);
            __syncwarp();
        }
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
    }
}

template <int NCOLS>
void launch_bulk_cols(dim3 grid, size_t smem, cudaStream_t st, const GemmDesc &d, const CUtensorMap &mh, const CUtensorMap &ml,
                      const i64 *rowA, const i64 *bslot, const float *img, float2 *C, int BNc, int S, int *err) {
    cudaFuncSetAttribute(tc_zgemm_bulk_kernel<NCOLS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc_zgemm_bulk_kernel<NCOLS><<<grid, TMA_THREADS, smem, st>>>(with_wait_limit(d), mh, ml, rowA, bslot, img, C, BNc, S, err);
}


// The timeout path of the tensor-core kernels on its own: one warp allocates TMEM, waits on an
// mbarrier that nothing arrives on with the given limit, records the timeout in *err, frees TMEM
// and returns.
__global__ void wait_selftest_kernel(unsigned long long limit_ns, int *err) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&slot)), "r"(32));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = slot;
    const bool ok = mbar_wait(&bar, 0, limit_ns);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32));
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

template <typename TA>
static int launch_tc_reg(const GemmDesc &d, const TA *A, const float2 *B, float2 *C, int *err, cudaStream_t st) {
    // complex N tile: N split evenly into tiles of at most 128 (256 real TMEM columns), each a multiple of 8
    const i64 ntiles = ceil_div(d.N, 128);
    const int BNc = (int)(ceil_div(ceil_div(d.N, ntiles), 8) * 8);
    const int NR = 2 * BNc;
    const size_t smem = tc_zgemm_smem_bytes(BNc);
    const dim3 grid((unsigned)ceil_div(d.N, BNc), (unsigned)ceil_div(d.M, BM), (unsigned)d.batch);
    if (NR <= 32)
        launch_cols<32, TA>(grid, smem, st, d, A, B, C, BNc, err);
    else if (NR <= 64)
        launch_cols<64, TA>(grid, smem, st, d, A, B, C, BNc, err);
    else if (NR <= 128)
        launch_cols<128, TA>(grid, smem, st, d, A, B, C, BNc, err);
    else
        launch_cols<256, TA>(grid, smem, st, d, A, B, C, BNc, err);
    return 1;
}
int launch_tc_zgemm(const GemmDesc &d, const float2 *A, const float2 *B, float2 *C, int *err, cudaStream_t st) {
    return launch_tc_reg<float2>(d, A, B, C, err, st);
}
int launch_tc_zgemm_a64(const GemmDesc &d, const double2 *A, const float2 *B, float2 *C, int *err, cudaStream_t st) {
    return launch_tc_reg<double2>(d, A, B, C, err, st);
}

// ----------------------------------------------------------------------------- host side of the TMA path
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *, const cuuint64_t *,
                                  const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct TcOperands {
    DBuf<float2> hi[NBUF], lo[NBUF];
    // (buffer, row length, box floats) -> hi, lo maps (box 32: 128-byte swizzle, 16: 64-byte swizzle)
    std::map<std::tuple<int, i64, int>, std::pair<CUtensorMap, CUtensorMap>> maps;
    DBuf<float> img;   // B' images of the bulk-fed kernel (grown on demand)
};

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

ccgf_status tc_prepare(ccgf_handle *h, cudaStream_t st, size_t reserve) {
    if (h->tc_ops) return CCGF_OK;
    TcOperands *T = new TcOperands();
    // A operands of the plain GEMM steps only (the tensor GEMMs of the density-fitting terms run on SIMT);
    // a block without hi / lo copies runs on the register-fed kernel
    for (int b = BUF_FOO; b < BUF_LD; ++b) {
        if (!h->Wf[b].p) continue;
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess || fr < (size_t)h->Wf[b].n * 16 + reserve) continue;
        ccgf_status s = dalloc(T->hi[b], h->Wf[b].n);
        if (s == CCGF_OK) s = dalloc(T->lo[b], h->Wf[b].n);
        if (s != CCGF_OK) {
            for (int c = 0; c < NBUF; ++c) { dfree(T->hi[c]); dfree(T->lo[c]); }
            delete T;
            return s;
        }
        const i64 n = h->Wf[b].n;
        i64 g = ceil_div(n, 256);
        tf32_split_kernel<<<(unsigned)(g > 152 * 16 ? 152 * 16 : g), 256, 0, st>>>(h->Wf[b].p, T->hi[b].p, T->lo[b].p, n);
        h->launches++;
    }
    h->tc_ops = T;
    CCGF_CUDA_TRY(cudaGetLastError());
    return CCGF_OK;
}

void tc_free(ccgf_handle *h) {
    TcOperands *T = (TcOperands *)h->tc_ops;
    if (!T) return;
    for (int c = 0; c < NBUF; ++c) {
        dfree(T->hi[c]);
        dfree(T->lo[c]);
    }
    dfree(T->img);
    delete T;
    h->tc_ops = nullptr;
}

// tensor maps over the hi / lo copies of buffer a_buf viewed as rows of 2 rsA floats
static bool tc_maps(ccgf_handle *h, int a_buf, i64 rsA, int box_floats, const CUtensorMap **mh, const CUtensorMap **ml) {
    TcOperands *T = (TcOperands *)h->tc_ops;
    if (!T || a_buf < BUF_FOO || a_buf >= NBUF || !T->hi[a_buf].p || rsA <= 0 || (rsA & 1)) return false;
    auto key = std::make_tuple(a_buf, rsA, box_floats);
    auto it = T->maps.find(key);
    if (it == T->maps.end()) {
        EncodeTiledFn enc = encode_fn();
        if (!enc) return false;
        const i64 rows = T->hi[a_buf].n / rsA;
        if (rows < 1 || rows > (1LL << 31) - 1) return false;
        cuuint64_t dims[2] = {(cuuint64_t)(2 * rsA), (cuuint64_t)rows};
        cuuint64_t strides[1] = {(cuuint64_t)(2 * rsA * sizeof(float))};
        cuuint32_t box[2] = {(cuuint32_t)box_floats, (cuuint32_t)BM};
        cuuint32_t estr[2] = {1, 1};
        const CUtensorMapSwizzle sw = box_floats == 32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
        std::pair<CUtensorMap, CUtensorMap> m;
        CUresult r1 = enc(&m.first, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)T->hi[a_buf].p, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        CUresult r2 = enc(&m.second, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)T->lo[a_buf].p, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r1 != CUDA_SUCCESS || r2 != CUDA_SUCCESS) return false;
        it = T->maps.emplace(key, m).first;
    }
    *mh = &it->second.first;
    *ml = &it->second.second;
    return true;
}

int launch_tc_zgemm_tma(ccgf_handle *h, int a_buf, const GemmDesc &d, const i64 *rowA, const float2 *B, float2 *C, int *err,
                        cudaStream_t st) {
    const CUtensorMap *mh, *ml;
    if (d.csA != 1 || !rowA || !tc_maps(h, a_buf, d.rsA, 2 * BKC, &mh, &ml)) return 0;
    const int BNc = d.N >= 128 ? 128 : (int)ceil_div(d.N, 8) * 8;
    const int NR = 2 * BNc;
    const size_t stage = (size_t)2 * BM * 2 * BKC * 4 + (size_t)2 * NR * 2 * BKC * 4;
    const size_t extra = 1024 + 8 * (3 * MAX_STAGES + 1) + 16;
    int S = (int)((227 * 1024 - extra - 1024) / stage);   // 1024: static shared memory of the kernel
    if (S > MAX_STAGES) S = MAX_STAGES;
    if (S < 2) return 0;
    const size_t smem = S * stage + extra;
    const dim3 grid((unsigned)ceil_div(d.N, BNc), (unsigned)ceil_div(d.M, BM), (unsigned)d.batch);
    if (NR <= 32)
        launch_tma_cols<32>(grid, smem, st, d, *mh, *ml, rowA, B, C, BNc, S, err);
    else if (NR <= 64)
        launch_tma_cols<64>(grid, smem, st, d, *mh, *ml, rowA, B, C, BNc, S, err);
    else if (NR <= 128)
        launch_tma_cols<128>(grid, smem, st, d, *mh, *ml, rowA, B, C, BNc, S, err);
    else
        launch_tma_cols<256>(grid, smem, st, d, *mh, *ml, rowA, B, C, BNc, S, err);
    return 1;
}

// Bulk-fed variant: B' image for the nslots distinct B blocks (bsrc: their offsets; bslot: slot of
// each (batch, reduction) entry, both device tables), then the GEMM. Returns the launch count, or
// 0 when the operand does not qualify (nothing launched).
int launch_tc_zgemm_bulk(ccgf_handle *h, int a_buf, const GemmDesc &d, const i64 *rowA, const i64 *bslot, const i64 *bsrc,
                         int nslots, const float2 *B, float2 *C, int *err, cudaStream_t st) {
    const CUtensorMap *mh, *ml;
    TcOperands *T = (TcOperands *)h->tc_ops;
    if (!T || d.csA != 1 || !rowA || !bslot || !bsrc || nslots < 1 || !tc_maps(h, a_buf, d.rsA, 2 * BKC3, &mh, &ml)) return 0;
    const int BNc = tc3_bn(d), NR = 2 * BNc;
    const int ntiles = (int)ceil_div(d.N, BNc), ktiles = (int)ceil_div(d.K, BKC3);
    const i64 img_floats = (i64)nslots * ntiles * ktiles * NR * 2 * (2 * BKC3);
    if (T->img.n < img_floats) {
        // grow the image buffer (synchronises: the previous image may still be in use)
        if (cudaStreamSynchronize(st) != cudaSuccess) return 0;
        dfree(T->img);
        if (dalloc(T->img, img_floats) != CCGF_OK) return 0;
    }
    const size_t stage = (size_t)2 * BM * 2 * BKC3 * 4 + (size_t)NR * 2 * (2 * BKC3) * 4;
    const size_t extra = 1024 + 8 * (2 * MAX_STAGES3 + 1) + 16;
    int S = (int)((227 * 1024 - extra - 1024) / stage);
    if (S > MAX_STAGES3) S = MAX_STAGES3;
    if (S < 2) return 0;
    const size_t smem = S * stage + extra;
    {
        const i64 total = (i64)nslots * ntiles * ktiles * (BNc / 4) * 16;
        i64 g = ceil_div(total, 256);
        bimage_kernel<<<(unsigned)(g > 152 * 32 ? 152 * 32 : g), 256, 0, st>>>(d, B, bsrc, nslots, BNc, ntiles, ktiles, T->img.p);
    }
    const dim3 grid((unsigned)ntiles, (unsigned)ceil_div(d.M, BM), (unsigned)d.batch);
    if (NR <= 32)
        launch_bulk_cols<32>(grid, smem, st, d, *mh, *ml, rowA, bslot, T->img.p, C, BNc, S, err);
    else if (NR <= 64)
        launch_bulk_cols<64>(grid, smem, st, d, *mh, *ml, rowA, bslot, T->img.p, C, BNc, S, err);
    else if (NR <= 128)
        launch_bulk_cols<128>(grid, smem, st, d, *mh, *ml, rowA, bslot, T->img.p, C, BNc, S, err);
    else
        launch_bulk_cols<256>(grid, smem, st, d, *mh, *ml, rowA, bslot, T->img.p, C, BNc, S, err);
    return 2;
}

void launch_wait_selftest(double limit_ms, int *err, cudaStream_t st) {
    wait_selftest_kernel<<<1, 32, 0, st>>>((unsigned long long)(limit_ms * 1e6), err);
}

// ----------------------------------------------------------------------------- FP64-accurate variant
// Complex FP64 GEMM on the tensor cores by exact slicing (after Ozaki et al., error-free
// transformation of matrix products by splitting each operand into slices whose products are
// exact): every FP64 value x of a row of A (column of B) with max |x| < 2^e is written as
//   x = 2^e * (s0 2^-8 + s1 2^-16 + s2 2^-24 + s3 2^-32 + s4 2^-40) + r,   |r| <= 2^(e-41),
// rounding to nearest at each step, so |s0| <= 256 and |s1..s4| <= 128. Integers of this size are
// exact in TF32, so are their products, and sums below 2^24 are exact in the FP32 accumulator of
// tcgen05.mma.kind::tf32. Per output
//   x*y = 2^(eA+eB) (T0 2^-16 + T1 2^-24 + T2 2^-32 + T 2^-16),
//   T0 = s0 t0, T1 = s0 t1 + s1 t0, T2 = s0 t2 + s1 t1 + s2 t0 (integers, exact over 128 real K),
//   T = sum over i + j in {3, 4} of (si 2^-8i)(tj 2^-8j) (below 2^-24 of the leading term, so the FP32
//   rounding of its accumulation is ~2^-48 of it); terms with i + j > 4 (< 2^-40) are dropped.
// Per 8 real K the CTA issues 15 MMAs into the four TMEM accumulators of one of two chunk buffers;
// every chunk of at most 128 real K within one reduction block is drained by the epilogue warps into
// FP32 double-word accumulators scaled by 2^(eA + eB) while the MMAs fill the other buffer. Operands:
// A as seven stored planes (s0, s1, s2 and s1 2^-8, s2 2^-16, s3 2^-24, s4 2^-32) of the FP64
// intermediate with one exponent per stored row, by TMA; B as the same seven planes of the
// 2x2-embedded B' tile with one exponent per (block, column), written by oz_bimage_kernel and fetched
// by one cp.async.bulk per stage. Error ~2^-41 of n max|a| max|b| (largest magnitudes of the row of A
// and the column of B).
namespace {

constexpr int OZ_PLANES = 7;
constexpr int OZ_CHUNK_STAGES = 8;         // 8 stages x 16 real K = 128: the exactness bound of T2
constexpr int OZ_MAX_STAGES = 3;

// exponent e with |x| < 2^e for every |x| <= amax (0 when amax = 0)
__device__ __forceinline__ int oz_exponent(double amax) {
    int e = 0;
    if (amax > 0.0) frexp(amax, &e);
    return e;
}
// the seven plane values of x (|x| < 2^e)
__device__ __forceinline__ void oz_slice(double x, int e, float (&p)[OZ_PLANES]) {
    double t = ldexp(x, 8 - e);   // |t| < 256
    const double s0 = rint(t);
    t = (t - s0) * 256.0;
    const double s1 = rint(t);
    t = (t - s1) * 256.0;
    const double s2 = rint(t);
    t = (t - s2) * 256.0;
    const double s3 = rint(t);
    t = (t - s3) * 256.0;
    const double s4 = rint(t);
    p[0] = (float)s0;
    p[1] = (float)s1;
    p[2] = (float)s2;
    p[3] = (float)(s1 * 0x1p-8);
    p[4] = (float)(s2 * 0x1p-16);
    p[5] = (float)(s3 * 0x1p-24);
    p[6] = (float)(s4 * 0x1p-32);
}
// 2^e as a double for |e| < 1000
__device__ __forceinline__ double oz_pow2(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

// planes of an FP64 buffer viewed as rows of rs complex: one block per row (grid-strided)
__global__ void oz_plane_kernel(const double2 *__restrict__ W, i64 rows, i64 rs, float2 *__restrict__ planes, i64 plane_stride,
                                int *__restrict__ rowexp) {
    __shared__ double red[256];
    for (i64 y = blockIdx.x; y < rows; y += gridDim.x) {
        const double2 *row = W + y * rs;
        double m = 0.0;
        for (i64 k = threadIdx.x; k < rs; k += blockDim.x) m = fmax(m, fmax(fabs(row[k].x), fabs(row[k].y)));
        red[threadIdx.x] = m;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
            __syncthreads();
        }
        const int e = oz_exponent(red[0]);
        __syncthreads();
        if (threadIdx.x == 0) rowexp[y] = e;
        for (i64 k = threadIdx.x; k < rs; k += blockDim.x) {
            float pr[OZ_PLANES], pi[OZ_PLANES];
            oz_slice(row[k].x, e, pr);
            oz_slice(row[k].y, e, pi);
#pragma unroll
            for (int q = 0; q < OZ_PLANES; ++q) planes[q * plane_stride + y * rs + k] = make_float2(pr[q], pi[q]);
        }
    }
}

// exponent of every (slot, column) of B over its K complex entries: one warp per (slot, column)
__global__ void oz_colexp_kernel(GemmDesc d, const double2 *__restrict__ B, const i64 *__restrict__ bsrc, int nslots,
                                 int *__restrict__ colexp) {
    const int lane = threadIdx.x & 31;
    const i64 nw = (i64)nslots * d.N;
    for (i64 w = ((i64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nw; w += ((i64)gridDim.x * blockDim.x) >> 5) {
        const int slot = (int)(w / d.N), n = (int)(w % d.N);
        const double2 *col = B + bsrc[slot] + (i64)n * d.csB;
        double m = 0.0;
        for (int k = lane; k < d.K; k += 32) {
            const double2 v = col[(i64)k * d.rsB];
            m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (lane == 0) colexp[w] = oz_exponent(m);
    }
}

// B' planes of the slots: per (slot, N tile, K tile) seven planes of NR rows x 16 real K in the
// canonical no-swizzle K-major layout (as bimage_kernel); thread = (slot, N tile, K tile, 4-column
// group t, k pair kp, column nl)
__global__ void oz_bimage_kernel(GemmDesc d, const double2 *__restrict__ B, const i64 *__restrict__ bsrc, const int *__restrict__ colexp,
                                 int nslots, int BNc, int ntiles, int ktiles, float *__restrict__ img) {
    const int NR = 2 * BNc;
    const i64 plane = (i64)NR * (2 * BKC3);
    const i64 chunk = OZ_PLANES * plane;
    const i64 per_tile = (i64)(BNc / 4) * 16;
    const i64 total = (i64)nslots * ntiles * ktiles * per_tile;
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (i64)gridDim.x * blockDim.x) {
        const int nl = (int)(i & 3), kp = (int)((i >> 2) & 3);
        i64 r = i >> 4;
        const int t = (int)(r % (BNc / 4));
        r /= (BNc / 4);
        const int kt = (int)(r % ktiles);
        r /= ktiles;
        const int nt = (int)(r % ntiles);
        const int slot = (int)(r / ntiles);
        const int n = nt * BNc + t * 4 + nl, k = kt * BKC3 + kp * 2;
        double2 v0 = make_double2(0.0, 0.0), v1 = v0;
        int e = 0;
        if (n < d.N) {
            const double2 *col = B + bsrc[slot] + (i64)n * d.csB;
            if (k < d.K) v0 = col[(i64)k * d.rsB];
            if (k + 1 < d.K) v1 = col[(i64)(k + 1) * d.rsB];
            e = colexp[(i64)slot * d.N + n];
        }
        float r0[OZ_PLANES], i0[OZ_PLANES], r1[OZ_PLANES], i1[OZ_PLANES];
        oz_slice(v0.x, e, r0);
        oz_slice(v0.y, e, i0);
        oz_slice(v1.x, e, r1);
        oz_slice(v1.y, e, i1);
        float *base = img + (((i64)slot * ntiles + nt) * ktiles + kt) * chunk;
        const int o_re = t * 128 + kp * 32 + nl * 8, o_im = o_re + 4;   // in floats: row 2n, row 2n+1
#pragma unroll
        for (int q = 0; q < OZ_PLANES; ++q) {
            float *p = base + q * plane;
            *(float4 *)(p + o_re) = make_float4(r0[q], -i0[q], r1[q], -i1[q]);
            *(float4 *)(p + o_im) = make_float4(i0[q], r0[q], i1[q], r1[q]);
        }
    }
}

// exact sum of two floats: s + e = a + b
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += (vh, vl) in double-word FP32 arithmetic
__device__ __forceinline__ void dw_add(float &hi, float &lo, float vh, float vl) {
    float s, e;
    two_sum(hi, vh, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, vl));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

}  // namespace

namespace {

// FP64-accurate complex GEMM (see above). NR = 2 BNc real columns (32 or 64); TMEM holds
// T0 / T1 / T2 / T of two chunk buffers at columns q * NR, q = 4 * buffer + accumulator.
template <int NR>
__global__ void __launch_bounds__(TMA_THREADS, 1)
    tc_zgemm_oz_kernel(GemmDesc d, const __grid_constant__ CUtensorMap m0_, const __grid_constant__ CUtensorMap m1_,
                       const __grid_constant__ CUtensorMap m2_, const __grid_constant__ CUtensorMap m3_,
                       const __grid_constant__ CUtensorMap m4_, const __grid_constant__ CUtensorMap m5_,
                       const __grid_constant__ CUtensorMap m6_,
                       const i64 *__restrict__ rowA, const int *__restrict__ rowexp, i64 arows, const i64 *__restrict__ bslot,
                       const float *__restrict__ img, const int *__restrict__ colexp, double2 *__restrict__ C, int S, int *err) {
    constexpr int BNc = NR / 2;
    constexpr uint32_t NCOLS = NR <= 32 ? 256 : 512;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    constexpr uint32_t a_bytes = BM * 2 * BKC3 * 4;                      // 8 KB per plane
    constexpr uint32_t b_plane = (uint32_t)NR * 2 * BKC3 * 4;            // NR x 16 floats
    constexpr uint32_t b_bytes = OZ_PLANES * b_plane;
    constexpr uint32_t stage_bytes = OZ_PLANES * a_bytes + b_bytes;
    uint64_t *full = (uint64_t *)(base + S * stage_bytes);
    uint64_t *empty = full + OZ_MAX_STAGES;
    uint64_t *cfull = empty + OZ_MAX_STAGES;   // [2] chunk accumulated
    uint64_t *cempty = cfull + 2;              // [2] chunk drained
    uint64_t *accum = cempty + 2;              // every MMA done
    uint32_t *tmem_slot = (uint32_t *)(accum + 1);
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.z, nt = blockIdx.x;
    const int mb = blockIdx.y * BM, n0 = nt * BNc;
    const int ktiles = (d.K + BKC3 - 1) / BKC3;
    const int ntiles = gridDim.x;
    const int total = d.nred * ktiles;
    const int cpr = (ktiles + OZ_CHUNK_STAGES - 1) / OZ_CHUNK_STAGES;   // chunks per reduction block
    const int nchunks = d.nred * cpr;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int p = 0; p < 2; ++p) {
            mbar_init(&cfull[p], 1);
            mbar_init(&cempty[p], 4);
        }
        mbar_init(accum, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)), "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    volatile int *abort_v = &abort_flag;

    if (warp == 0) {
        if (lane == 0) {
            const CUtensorMap *maps[OZ_PLANES] = {&m0_, &m1_, &m2_, &m3_, &m4_, &m5_, &m6_};
            int issued = 0;
            for (int kt = 0; kt < total; ++kt) {
                const int s = kt % S;
                if (kt >= S && !mbar_wait_or_abort(&empty[s], ((kt / S) - 1) & 1, abort_v, d.wait_ns)) {
                    atomicExch(err, 1);
                    *abort_v = 1;
                    break;
                }
                const int r = kt / ktiles, kk = kt % ktiles;
                const i64 br = (i64)b * d.nred + r;
                const int y = (int)rowA[br] + mb;
                unsigned char *sA = base + s * stage_bytes;
                const float *src = img + (((i64)bslot[br] * ntiles + nt) * ktiles + kk) * ((i64)b_bytes / 4);
                mbar_expect_tx(&full[s], stage_bytes);
#pragma unroll
                for (int q = 0; q < OZ_PLANES; ++q) tma_load_2d(smem_u32(sA + q * a_bytes), maps[q], 2 * kk * BKC3, y, &full[s]);
                bulk_load(smem_u32(sA + OZ_PLANES * a_bytes), src, b_bytes, &full[s]);
                issued = kt + 1;
            }
            for (int kt = issued - S > 0 ? issued - S : 0; kt < issued; ++kt)
                if (!mbar_wait(&full[kt % S], (kt / S) & 1, d.wait_ns)) atomicExch(err, 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = make_idesc(NR);
            // (A plane, B plane, accumulator) of the 15 products: T0 = s0 t0; T1 = s0 t1 + s1 t0;
            // T2 = s0 t2 + s1 t1 + s2 t0; T = the nine scaled products with i + j = 3, 4
            const int pa[15] = {0, 0, 1, 0, 1, 2, 0, 3, 4, 5, 0, 3, 4, 5, 6};
            const int pb[15] = {0, 1, 0, 2, 1, 0, 5, 4, 3, 0, 6, 5, 4, 3, 0};
            const int pc[15] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3, 3, 3};
            int issued = 0, c = -1;
            for (int kt = 0; kt < total; ++kt) {
                const int s = kt % S;
                const int kk = kt % ktiles;
                const bool cstart = kk % OZ_CHUNK_STAGES == 0;
                const bool cend = kk % OZ_CHUNK_STAGES == OZ_CHUNK_STAGES - 1 || kk == ktiles - 1;
                if (cstart) {
                    ++c;
                    if (c >= 2 && !mbar_wait_or_abort(&cempty[c & 1], ((c >> 1) - 1) & 1, abort_v, d.wait_ns)) {
                        atomicExch(err, 1);
                        *abort_v = 1;
                        break;
                    }
                }
                if (!mbar_wait_or_abort(&full[s], (kt / S) & 1, abort_v, d.wait_ns)) {
                    atomicExch(err, 1);
                    *abort_v = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = smem_u32(base + s * stage_bytes), sb = sa + OZ_PLANES * a_bytes;
                const uint32_t tacc = tmem + (uint32_t)((c & 1) * 4 * NR);
#pragma unroll
                for (int ks = 0; ks < (2 * BKC3) / 8; ++ks) {
#pragma unroll
                    for (int q = 0; q < 15; ++q) {
                        const uint64_t da = make_desc_sw64(sa + pa[q] * a_bytes + ks * 32);
                        const uint64_t db = make_desc_k16(sb + pb[q] * b_plane + ks * 256);
                        // the first product into each accumulator of a chunk overwrites it
                        const bool first = cstart && ks == 0 && (q == 0 || q == 1 || q == 3 || q == 6);
                        mma_tf32(tacc + (uint32_t)(pc[q] * NR), da, db, idesc, first ? 0u : 1u);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&empty[s]))
                             : "memory");
                if (cend)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&cfull[c & 1]))
                                 : "memory");
                issued = kt + 1;
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(accum))
                         : "memory");
            if (issued < total) *abort_v = 1;
        }
    } else {
        // epilogue: thread = output row (TMEM lane quarter * 32 + lane), NR real columns in double-word FP32
        const int quarter = warp & 3;
        const int m = mb + quarter * 32 + lane;
        float ah[NR], al[NR];
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            ah[j] = 0.f;
            al[j] = 0.f;
        }
        bool ok = true;
        for (int c = 0; c < nchunks && ok; ++c) {
            const int r = c / cpr;
            ok = mbar_wait_or_abort(&cfull[c & 1], (c >> 1) & 1, abort_v, d.wait_ns);
            if (!__all_sync(0xffffffffu, ok)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const i64 br = (i64)b * d.nred + r;
            const i64 ya = rowA[br] + m;
            const int ea = ya < arows ? rowexp[ya] : 0;
            const int *ce = colexp + (i64)bslot[br] * d.N;
            const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((c & 1) * 4 * NR);
#pragma unroll
            for (int c0 = 0; c0 < NR; c0 += 8) {
                uint32_t v0[8], v1[8], v2[8], v3[8];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(v0[0]), "=r"(v0[1]), "=r"(v0[2]), "=r"(v0[3]), "=r"(v0[4]), "=r"(v0[5]), "=r"(v0[6]), "=r"(v0[7])
                             : "r"(tbase + (uint32_t)c0));
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(v1[0]), "=r"(v1[1]), "=r"(v1[2]), "=r"(v1[3]), "=r"(v1[4]), "=r"(v1[5]), "=r"(v1[6]), "=r"(v1[7])
                             : "r"(tbase + (uint32_t)(NR + c0)));
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(v2[0]), "=r"(v2[1]), "=r"(v2[2]), "=r"(v2[3]), "=r"(v2[4]), "=r"(v2[5]), "=r"(v2[6]), "=r"(v2[7])
                             : "r"(tbase + (uint32_t)(2 * NR + c0)));
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(v3[0]), "=r"(v3[1]), "=r"(v3[2]), "=r"(v3[3]), "=r"(v3[4]), "=r"(v3[5]), "=r"(v3[6]), "=r"(v3[7])
                             : "r"(tbase + (uint32_t)(3 * NR + c0)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int n = n0 + (c0 + j) / 2;
                    const int eb = n < d.N ? ce[n] : 0;
                    // value in units of 2^-32: T0 2^16 + T1 2^8 + T2 + T 2^16 as a double word
                    float vh, vl, s2, e2;
                    two_sum(__uint_as_float(v0[j]) * 65536.f, __uint_as_float(v1[j]) * 256.f, vh, vl);
                    two_sum(vh, __uint_as_float(v2[j]), s2, e2);
                    vh = s2;
                    vl = __fadd_rn(__fadd_rn(vl, e2), __uint_as_float(v3[j]) * 65536.f);
                    // scale by 2^(ea + eb - 32): exact inside the FP32 range (below it the term is dropped,
                    // above it the result becomes infinite, so that no wrong finite value is written)
                    const int ex = ea + eb - 32 + 127;
                    const float sc = ex < 1 ? 0.f : (ex > 254 ? __int_as_float(0x7f800000) : __int_as_float(ex << 23));
                    dw_add(ah[c0 + j], al[c0 + j], vh * sc, vl * sc);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&cempty[c & 1]);
        }
        if (!ok) atomicExch(err, 1);
        if (__all_sync(0xffffffffu, ok) && !*abort_v && m < d.M) {
            const double ax = d.alpha.x, ay = d.alpha.y, bx = d.beta.x, by = d.beta.y;
            const bool use_beta = (bx != 0.0 || by != 0.0);
            double2 *Cb = C + d.offC[b];
#pragma unroll
            for (int q = 0; q < BNc; ++q) {
                const int n = n0 + q;
                if (n >= d.N) continue;
                const double re = (double)ah[2 * q] + (double)al[2 * q], im = (double)ah[2 * q + 1] + (double)al[2 * q + 1];
                double2 *cp = Cb + (i64)m * d.rsC + (i64)n * d.csC;
                double2 o;
                o.x = ax * re - ay * im;
                o.y = ax * im + ay * re;
                if (use_beta) {
                    const double2 cv = *cp;
                    o.x += bx * cv.x - by * cv.y;
                    o.y += bx * cv.y + by * cv.x;
                }
                *cp = o;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        if (*abort_v) {
            if (!mbar_wait(accum, 0, d.wait_ns)) atomicExch(err, 1);
            __syncwarp();
        }
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
    }
}

}  // namespace

// ----------------------------------------------------------------------------- host side of the FP64-accurate path
// Seven planes and the row exponents of an intermediate, made on first use for one row length
// (the view its GEMMs use), only while the device keeps its reserve free afterwards.
struct OzPlanes {
    i64 rs = 0, rows = 0;
    DBuf<float2> planes;   // [7][pstride]
    DBuf<int> rowexp;      // [rows]
    CUtensorMap maps[OZ_PLANES];
};
struct OzState {
    OzPlanes *p[NBUF] = {};
    bool refused[NBUF] = {};
    DBuf<float> img;
    DBuf<int> colexp;
};

static OzState *oz_state(ccgf_handle *h) {
    if (!h->oz_ops) h->oz_ops = new OzState();
    return (OzState *)h->oz_ops;
}

void oz_free(ccgf_handle *h) {
    OzState *O = (OzState *)h->oz_ops;
    if (!O) return;
    for (int b = 0; b < NBUF; ++b) delete O->p[b];
    delete O;
    h->oz_ops = nullptr;
}

static const OzPlanes *oz_planes(ccgf_handle *h, int a_buf, i64 rs, cudaStream_t st) {
    if (a_buf < BUF_FOO || a_buf >= NBUF || !h->W[a_buf].p || rs <= 0 || (rs & 1)) return nullptr;
    OzState *O = oz_state(h);
    if (O->p[a_buf]) return O->p[a_buf]->rs == rs ? O->p[a_buf] : nullptr;
    if (O->refused[a_buf]) return nullptr;
    // planes 16-byte aligned: stride rounded up to an even number of complex elements
    const i64 n = h->W[a_buf].n, rows = n / rs, pstride = (n + 1) & ~(i64)1;
    EncodeTiledFn enc = encode_fn();
    size_t fr = 0, tot = 0;
    const size_t bytes = (size_t)OZ_PLANES * pstride * sizeof(float2) + (size_t)rows * sizeof(int);
    if (!enc || rows < 1 || rows > (1LL << 31) - 1 || cudaMemGetInfo(&fr, &tot) != cudaSuccess || fr < bytes + h->oz_reserve) {
        O->refused[a_buf] = true;
        return nullptr;
    }
    OzPlanes *P = new OzPlanes();
    P->rs = rs;
    P->rows = rows;
    if (dalloc(P->planes, OZ_PLANES * pstride) != CCGF_OK || dalloc(P->rowexp, rows) != CCGF_OK) {
        delete P;
        O->refused[a_buf] = true;
        return nullptr;
    }
    const unsigned g = (unsigned)std::min<i64>(rows, 152 * 8);
    oz_plane_kernel<<<g, 256, 0, st>>>(h->W[a_buf].p, rows, rs, P->planes.p, pstride, P->rowexp.p);
    h->launches++;
    if (cudaGetLastError() != cudaSuccess) {
        delete P;
        O->refused[a_buf] = true;
        return nullptr;
    }
    cuuint64_t dims[2] = {(cuuint64_t)(2 * rs), (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(2 * rs * sizeof(float))};
    cuuint32_t box[2] = {(cuuint32_t)(2 * BKC3), (cuuint32_t)BM};
    cuuint32_t estr[2] = {1, 1};
    for (int q = 0; q < OZ_PLANES; ++q) {
        CUresult r = enc(&P->maps[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)(P->planes.p + (i64)q * pstride), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            delete P;
            O->refused[a_buf] = true;
            return nullptr;
        }
    }
    O->p[a_buf] = P;
    return P;
}

template <int NR>
static cudaError_t launch_oz_cols(dim3 grid, size_t smem, cudaStream_t st, const GemmDesc &d, const OzPlanes *P, const i64 *rowA,
                                  const i64 *bslot, const float *img, const int *colexp, double2 *C, int S, int *err) {
    cudaError_t e = cudaFuncSetAttribute(tc_zgemm_oz_kernel<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tc_zgemm_oz_kernel<NR><<<grid, TMA_THREADS, smem, st>>>(with_wait_limit(d), P->maps[0], P->maps[1], P->maps[2], P->maps[3],
                                                           P->maps[4], P->maps[5], P->maps[6], rowA, P->rowexp.p, P->rows, bslot, img,
                                                           colexp, C,
                                                           S, err);
    return cudaGetLastError();
}

// a launch the sliced path could not make: the caller falls back to FP64 SIMT; the first few are
// reported on stderr with the GEMM's shape (they indicate a shape this path does not handle)
static int oz_launch_failed(const char *what, cudaError_t e, const GemmDesc &d, size_t smem) {
    static std::atomic<int> reported{0};
    if (reported.fetch_add(1) < 4)
        fprintf(stderr, "ccgf: sliced FP64 GEMM not used (%s: %s; M %d N %d K %d nred %d batch %d smem %zu)\n", what,
                cudaGetErrorString(e), d.M, d.N, d.K, d.nred, d.batch, smem);
    return 0;
}

bool tc_zgemm_oz_supported(const GemmDesc &d) { return d.M > 0 && d.N > 0 && d.K > 0 && d.csA == 1 && (d.rsA % 2) == 0; }

int launch_tc_zgemm_oz(ccgf_handle *h, int a_buf, const GemmDesc &d, const i64 *rowA, const i64 *bslot, const i64 *bsrc, int nslots,
                       const double2 *B, double2 *C, int *err, cudaStream_t st) {
    if (!tc_zgemm_oz_supported(d) || !rowA || !bslot || !bsrc || nslots < 1 || !err) return 0;
    const OzPlanes *P = oz_planes(h, a_buf, d.rsA, st);
    if (!P) return 0;
    OzState *O = oz_state(h);
    const int BNc = d.N <= 16 ? 16 : 32, NR = 2 * BNc;
    const int ntiles = (int)ceil_div(d.N, BNc), ktiles = (int)ceil_div(d.K, BKC3);
    const i64 img_floats = (i64)nslots * ntiles * ktiles * OZ_PLANES * NR * (2 * BKC3);
    const i64 ncol = (i64)nslots * d.N;
    if (O->img.n < img_floats || O->colexp.n < ncol) {
        // grow (synchronises: the previous image may still be in use)
        if (cudaStreamSynchronize(st) != cudaSuccess) return 0;
        if (O->img.n < img_floats) {
            dfree(O->img);
            if (dalloc(O->img, img_floats) != CCGF_OK) return 0;
        }
        if (O->colexp.n < ncol) {
            dfree(O->colexp);
            if (dalloc(O->colexp, ncol) != CCGF_OK) return 0;
        }
    }
    const size_t stage = (size_t)OZ_PLANES * BM * 2 * BKC3 * 4 + (size_t)OZ_PLANES * NR * 2 * BKC3 * 4;
    const size_t extra = 1024 + 8 * (2 * OZ_MAX_STAGES + 5) + 16;
    int S = (int)((227 * 1024 - extra) / stage);
    if (S > OZ_MAX_STAGES) S = OZ_MAX_STAGES;
    if (S < 2) return 0;
    const size_t smem = S * stage + extra;
    const dim3 grid((unsigned)ntiles, (unsigned)ceil_div(d.M, BM), (unsigned)d.batch);
    if (grid.y > 65535 || grid.z > 65535) return 0;
    {
        if (cudaPeekAtLastError() != cudaSuccess) return 0;   // an earlier error is left to its caller
        const i64 g = ceil_div(ncol * 32, 256);
        oz_colexp_kernel<<<(unsigned)(g > 152 * 16 ? 152 * 16 : g), 256, 0, st>>>(d, B, bsrc, nslots, O->colexp.p);
        const i64 total = (i64)nslots * ntiles * ktiles * (BNc / 4) * 16;
        const i64 g2 = ceil_div(total, 256);
        oz_bimage_kernel<<<(unsigned)(g2 > 152 * 32 ? 152 * 32 : g2), 256, 0, st>>>(d, B, bsrc, O->colexp.p, nslots, BNc, ntiles,
                                                                                    ktiles, O->img.p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return oz_launch_failed("B image", e, d, smem);
    }
    const cudaError_t e = NR == 32 ? launch_oz_cols<32>(grid, smem, st, d, P, rowA, bslot, O->img.p, O->colexp.p, C, S, err)
                                   : launch_oz_cols<64>(grid, smem, st, d, P, rowA, bslot, O->img.p, O->colexp.p, C, S, err);
    if (e != cudaSuccess) return oz_launch_failed("GEMM", e, d, smem);
    return 3;
}
