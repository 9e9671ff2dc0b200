// Generic device kernels: batched complex GEMM (FP64 / FP32 SIMT), batched strided
// permute-add, layout transposes, plus small shared helpers of the library.
#include "ccgf_internal.h"
#include <atomic>
#include <mutex>
#include <cmath>

static thread_local std::string g_last_error;
void set_last_error(const std::string &msg) { g_last_error = msg; }
extern "C" const char *ccgf_last_error(void) { return g_last_error.c_str(); }

// Host-side failure injection for the error-path tests: after `g_fail_after` more successful
// allocations, every dalloc_bytes reports an out-of-memory error without calling cudaMalloc.
static std::atomic<long long> g_fail_after{-1};
extern "C" void ccgf_inject_alloc_failure(long long after) { g_fail_after.store(after); }

ccgf_status dalloc_bytes(void **p, size_t bytes) {
    long long left = g_fail_after.load();
    while (left >= 0) {
        if (left == 0) {
            *p = nullptr;
            set_last_error("cudaMalloc(" + std::to_string(bytes) + "): injected out-of-memory failure");
            return CCGF_ERR_OOM;
        }
        if (g_fail_after.compare_exchange_weak(left, left - 1)) break;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        set_last_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? CCGF_ERR_OOM : CCGF_ERR_CUDA;
    }
    return CCGF_OK;
}

void KMeshH::init(const int kmesh[3]) {
    n[0] = kmesh[0];
    n[1] = kmesh[1];
    n[2] = kmesh[2];
    nk = n[0] * n[1] * n[2];
    add.assign(nk * nk, 0);
    sub.assign(nk * nk, 0);
    for (int x = 0; x < nk; ++x) {
        int xv[3] = {x / (n[1] * n[2]), (x / n[2]) % n[1], x % n[2]};
        for (int y = 0; y < nk; ++y) {
            int yv[3] = {y / (n[1] * n[2]), (y / n[2]) % n[1], y % n[2]};
            int sa[3], sd[3];
            for (int d = 0; d < 3; ++d) {
                sa[d] = (xv[d] + yv[d]) % n[d];
                sd[d] = ((xv[d] - yv[d]) % n[d] + n[d]) % n[d];
            }
            add[x * nk + y] = (sa[0] * n[1] + sa[1]) * n[2] + sa[2];
            sub[x * nk + y] = (sd[0] * n[1] + sd[1]) * n[2] + sd[2];
        }
    }
}

// ----------------------------------------------------------------------------- complex helpers
template <typename T> __device__ __forceinline__ T cz();
template <> __device__ __forceinline__ double2 cz<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 cz<float2>() { return make_float2(0.f, 0.f); }

template <typename T, typename S> __device__ __forceinline__ void cfma(T &acc, const T a, const T b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// ----------------------------------------------------------------------------- batched GEMM
// (TY TM) x (TX TN) output tile per CTA, 256 threads as TY rows x TX = 256 / TY columns, TM x TN
// complex outputs per thread (rows ty + TY i, columns tx + TX j), K staged through shared memory
// 16 at a time. Loads pick the coalesced mapping from whichever operand stride is 1. Out-of-range
// rows / columns of a tile are zero-filled on load and masked on store. The launcher picks
// (TM, TN, TY) per GEMM to keep tile padding small (e.g. 88 rows -> 2 x 48 or 1 x 88).
template <typename R, int TM, int TN, int TY = 16>
__global__ void __launch_bounds__(256) zgemm_kernel(GemmDesc d, const typename cvec<R>::T *__restrict__ A,
                                                    const typename cvec<R>::T *__restrict__ B,
                                                    typename cvec<R>::T *__restrict__ C, int ksplit, int kchunk,
                                                    typename cvec<R>::T *__restrict__ work) {
    typedef typename cvec<R>::T T;
    constexpr int TX = 256 / TY;
    constexpr int BM = TY * TM, BN = TX * TN, BK = 16;
    constexpr int NLA = (BM * BK + 255) / 256, NLB = (BN * BK + 255) / 256;   // tile loads per thread
    __shared__ T As[BK][BM];
    __shared__ T Bs[BK][BN];
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const T alpha = {(R)d.alpha.x, (R)d.alpha.y};
    const T beta = {(R)d.beta.x, (R)d.beta.y};
    const bool use_beta = (d.beta.x != 0.0 || d.beta.y != 0.0);
    for (int bz = blockIdx.z; bz < d.batch * ksplit; bz += gridDim.z) {
        const int b = bz / ksplit, ks = bz % ksplit;
        // a split covers a K range of every momentum block (nred = 1), or whole momentum blocks
        // [rbeg, rend) (nred > 1, kchunk = K; rchunk blocks per split)
        const int rchunk = d.nred > 1 ? (d.nred + ksplit - 1) / ksplit : 1;
        const int rbeg = d.nred > 1 ? ks * rchunk : 0, rend = d.nred > 1 ? min(d.nred, rbeg + rchunk) : 1;
        const int kbeg = d.nred > 1 ? 0 : ks * kchunk, kend = d.nred > 1 ? d.K : min(d.K, kbeg + kchunk);
        T acc[TM][TN];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = cz<T>();
        for (int r = rbeg; r < rend; ++r) {
            const T *Ab = A + d.offA[(i64)b * d.nred + r];
            const T *Bb = B + d.offB[(i64)b * d.nred + r];
            for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
                for (int s = 0; s < NLA; ++s) {
                    int l = tid + 256 * s, i, kk;
                    if (BM * BK % 256 != 0 && l >= BM * BK) break;
                    if (d.csA == 1) { kk = l & 15; i = l >> 4; } else { i = l % BM; kk = l / BM; }
                    int m = m0 + i, k = k0 + kk;
                    As[kk][i] = (m < d.M && k < kend) ? Ab[(i64)m * d.rsA + (i64)k * d.csA] : cz<T>();
                }
#pragma unroll
                for (int s = 0; s < NLB; ++s) {
                    int l = tid + 256 * s, nn, kk;
                    if (BN * BK % 256 != 0 && l >= BN * BK) break;
                    if (d.csB == 1) { nn = l % BN; kk = l / BN; } else { kk = l & 15; nn = l >> 4; }
                    int n = n0 + nn, k = k0 + kk;
                    Bs[kk][nn] = (n < d.N && k < kend) ? Bb[(i64)k * d.rsB + (i64)n * d.csB] : cz<T>();
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < BK; ++kk) {
                    T a[TM], bb[TN];
#pragma unroll
                    for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + TY * i];
#pragma unroll
                    for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx + TX * j];
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) cfma<T, R>(acc[i][j], a[i], bb[j]);
                }
                __syncthreads();
            }
        }
        if (ksplit > 1) {
            // raw partial sums to work[b][ks][M][N]; zgemm_splitk_reduce applies alpha and beta
            T *Wb = work + ((i64)b * ksplit + ks) * (i64)d.M * d.N;
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                int m = m0 + ty + TY * i;
                if (m >= d.M) continue;
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    int n = n0 + tx + TX * j;
                    if (n < d.N) Wb[(i64)m * d.N + n] = acc[i][j];
                }
            }
            continue;
        }
        T *Cb = C + d.offC[b];
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            int m = m0 + ty + TY * i;
            if (m >= d.M) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                int n = n0 + tx + TX * j;
                if (n >= d.N) continue;
                T *c = Cb + (i64)m * d.rsC + (i64)n * d.csC;
                T v;
                v.x = alpha.x * acc[i][j].x - alpha.y * acc[i][j].y;
                v.y = alpha.x * acc[i][j].y + alpha.y * acc[i][j].x;
                if (use_beta) {
                    T o = *c;
                    v.x += beta.x * o.x - beta.y * o.y;
                    v.y += beta.x * o.y + beta.y * o.x;
                }
                *c = v;
            }
        }
    }
}

template <typename R>
__global__ void zgemm_splitk_reduce(GemmDesc d, int ksplit, const typename cvec<R>::T *__restrict__ work,
                                    typename cvec<R>::T *__restrict__ C) {
    typedef typename cvec<R>::T T;
    const i64 mn = (i64)d.M * d.N;
    const bool use_beta = (d.beta.x != 0.0 || d.beta.y != 0.0);
    for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t < mn * d.batch; t += (i64)gridDim.x * blockDim.x) {
        const int b = (int)(t / mn);
        const i64 e = t - (i64)b * mn;
        const int m = (int)(e / d.N), n = (int)(e - (i64)m * d.N);
        R sx = 0, sy = 0;
        for (int s = 0; s < ksplit; ++s) {
            T p = work[((i64)b * ksplit + s) * mn + e];
            sx += p.x;
            sy += p.y;
        }
        T *c = C + d.offC[b] + (i64)m * d.rsC + (i64)n * d.csC;
        T v;
        v.x = (R)d.alpha.x * sx - (R)d.alpha.y * sy;
        v.y = (R)d.alpha.x * sy + (R)d.alpha.y * sx;
        if (use_beta) {
            T o = *c;
            v.x += (R)d.beta.x * o.x - (R)d.beta.y * o.y;
            v.y += (R)d.beta.x * o.y + (R)d.beta.y * o.x;
        }
        *c = v;
    }
}

// Per-thread tile shapes available to the launcher (rows x columns of complex outputs).
struct TileShape {
    int tm, tn, ty;   // per-thread rows, columns; thread rows of the CTA (16 or 8)
    i64 bm() const { return (i64)ty * tm; }
    i64 bn() const { return (i64)(256 / ty) * tn; }
};
// (the 9th-12th serve contractions with few rows or columns: an o x o Fock block, a single
// right-hand-side column block, ...; the last two have 8-row granularity: 88 or 24 rows exactly)
static const TileShape kShapes[] = {{4, 4, 16}, {3, 4, 16}, {2, 4, 16}, {4, 3, 16}, {4, 2, 16}, {4, 7, 16}, {3, 7, 16},
                                    {2, 7, 16}, {2, 2, 16}, {1, 4, 16}, {1, 7, 16}, {1, 2, 16}, {11, 2, 8}, {3, 2, 8}};

// Shape with the least padded work divided by the wave efficiency (whole waves of one CTA per
// SM), with a slight preference for larger tiles (higher register reuse).
int zgemm_tile_count() { return (int)(sizeof(kShapes) / sizeof(kShapes[0])); }

static TileShape pick_shape(const GemmDesc &d) {
    if (d.tile > 0 && d.tile <= zgemm_tile_count()) return kShapes[d.tile - 1];
    TileShape best = kShapes[0];
    double best_cost = 1e300;
    for (const TileShape &s : kShapes) {
        const i64 bm = s.bm(), bn = s.bn();
        const double padded = (double)ceil_div(d.M, bm) * bm * (double)ceil_div(d.N, bn) * bn;
        const double ctas = (double)ceil_div(d.M, bm) * ceil_div(d.N, bn) * d.batch;
        const double waves = ctas / 152.0;
        const double wave_eff = waves >= 1.0 ? waves / std::ceil(waves) : waves;
        const double cost = padded / wave_eff * (1.0 + 0.02 * (16.0 / (s.tm * s.tn * (16.0 / s.ty))));
        if (cost < best_cost) {
            best_cost = cost;
            best = s;
        }
    }
    return best;
}

// 1-based index of the tile the launcher's model picks for d
int zgemm_model_tile(const GemmDesc &d) {
    const TileShape s = pick_shape(d);
    for (int i = 0; i < zgemm_tile_count(); ++i)
        if (kShapes[i].tm == s.tm && kShapes[i].tn == s.tn && kShapes[i].ty == s.ty) return i + 1;
    return 0;
}

int zgemm_ksplit(const GemmDesc &d) {
    if (d.ksplit > 0) {
        // explicit split: over the momentum blocks when there are several (every split non-empty),
        // else over K with at least 16 per slice
        if (d.nred > 1) {
            const int rchunk = (int)ceil_div(d.nred, d.ksplit);
            return (int)ceil_div(d.nred, rchunk);
        }
        i64 kmax = ceil_div(d.K, 16);
        return (int)(d.ksplit < kmax ? d.ksplit : kmax);
    }
    // Enough CTAs to cover the SMs twice; every split keeps at least 8 k-tiles of work.
    const TileShape s = pick_shape(d);
    const i64 tiles = ceil_div(d.M, s.bm()) * ceil_div(d.N, s.bn()) * (i64)d.batch;
    if (tiles >= 304 || d.nred != 1) return 1;
    i64 k = ceil_div(304, tiles);
    i64 kmax = d.K / 128;
    if (k > kmax) k = kmax;
    return (int)(k < 1 ? 1 : k);
}
// Split (2..8) that best fills whole waves of one CTA per SM for the given tile: over whole momentum
// blocks when there are several (only splits that divide them evenly into non-empty groups), else
// over K with at least 32 per slice; 1 when no split improves the wave efficiency by more than 5 %.
int zgemm_wave_split(const GemmDesc &d, int tile) {
    GemmDesc e = d;
    e.tile = tile;
    const TileShape s = pick_shape(e);
    const double ctas = (double)ceil_div(d.M, s.bm()) * ceil_div(d.N, s.bn()) * d.batch;
    auto eff = [&](int k) {
        const double w = ctas * k / 152.0;
        return w / std::ceil(w);
    };
    // effective number of splits: over momentum blocks (nred > 1) or over K (>= 32 per slice)
    auto splits = [&](int k) -> int {
        if (d.nred > 1) return (int)ceil_div(d.nred, ceil_div(d.nred, k));
        return d.K / k >= 32 ? k : 0;
    };
    int best = 1;
    for (int k = 2; k <= 8; ++k) {
        const int e = splits(k);
        if (e < 2 || e != k) continue;
        if (eff(k) > eff(best) + 1e-12) best = k;
    }
    return eff(best) > 1.05 * eff(1) ? best : 1;
}
i64 zgemm_workspace_elems(const GemmDesc &d) {
    int s = zgemm_ksplit(d);
    return s > 1 ? (i64)s * d.M * d.N * d.batch : 0;
}

template <typename R, int TM, int TN, int TY = 16>
static void launch_shape(const GemmDesc &d, const typename cvec<R>::T *A, const typename cvec<R>::T *B, typename cvec<R>::T *C,
                         cudaStream_t st, int ks, int kchunk, typename cvec<R>::T *work) {
    i64 z = (i64)d.batch * ks;
    dim3 grid((unsigned)ceil_div(d.N, (256 / TY) * TN), (unsigned)ceil_div(d.M, TY * TM), (unsigned)(z < 65535 ? z : 65535));
    zgemm_kernel<R, TM, TN, TY><<<grid, 256, 0, st>>>(d, A, B, C, ks, kchunk, work);
}

template <typename R>
int launch_zgemm(const GemmDesc &d, const typename cvec<R>::T *A, const typename cvec<R>::T *B,
                 typename cvec<R>::T *C, cudaStream_t st, typename cvec<R>::T *work, i64 work_elems) {
    if (d.batch <= 0 || d.M <= 0 || d.N <= 0) return 0;
    int ks = zgemm_ksplit(d);
    if (ks > 1 && (work == nullptr || work_elems < zgemm_workspace_elems(d))) ks = 1;
    int kchunk = d.K;
    if (ks > 1 && d.nred == 1) {
        kchunk = (int)(ceil_div(ceil_div(d.K, ks), 16) * 16);
        ks = (int)ceil_div(d.K, kchunk);
    }
    const TileShape s = pick_shape(d);
    if (s.tm == 4 && s.tn == 4) launch_shape<R, 4, 4>(d, A, B, C, st, ks, kchunk, work);
    else if (s.tm == 3 && s.tn == 4) launch_shape<R, 3, 4>(d, A, B, C, st, ks, kchunk, work);
    else if (s.tm == 2 && s.tn == 4) launch_shape<R, 2, 4>(d, A, B, C, st, ks, kchunk, work);
    else if (s.tm == 4 && s.tn == 3) launch_shape<R, 4, 3>(d, A, B, C, st, ks, kchunk, work);
    else if (s.tm == 4 && s.tn == 2) launch_shape<R, 4, 2>(d, A, B, C, st, ks, kchunk, work);
    else if (s.tm == 4 && s.tn == 7) launch_shape<R, 4, 7>(d, A, B, C, st, ks, kchunk, work);
    else if (s.tm == 3 && s.tn == 7) launch_shape<R, 3, 7>(d, A, B, C, st, ks, kchunk, work);
    else if (s.tm == 2 && s.tn == 7) launch_shape<R, 2, 7>(d, A, B, C, st, ks, kchunk, work);
    else if (s.tm == 2 && s.tn == 2) launch_shape<R, 2, 2>(d, A, B, C, st, ks, kchunk, work);
    else if (s.tm == 1 && s.tn == 4) launch_shape<R, 1, 4>(d, A, B, C, st, ks, kchunk, work);
    else if (s.tm == 1 && s.tn == 7) launch_shape<R, 1, 7>(d, A, B, C, st, ks, kchunk, work);
    else if (s.tm == 11 && s.tn == 2 && s.ty == 8) launch_shape<R, 11, 2, 8>(d, A, B, C, st, ks, kchunk, work);
    else if (s.tm == 3 && s.tn == 2 && s.ty == 8) launch_shape<R, 3, 2, 8>(d, A, B, C, st, ks, kchunk, work);
    else launch_shape<R, 1, 2>(d, A, B, C, st, ks, kchunk, work);
    if (ks > 1) {
        i64 n = (i64)d.M * d.N * d.batch;
        i64 g = ceil_div(n, 256);
        zgemm_splitk_reduce<R><<<(unsigned)(g > 4096 ? 4096 : g), 256, 0, st>>>(d, ks, work, C);
        return 2;
    }
    return 1;
}

// Contractions with at most 8 rows and a short reduction (an o x o Fock block applied to every
// column, for instance) are bound by streaming B and C: one thread per output column keeps the
// M partial sums in registers and reads each B element once; A (at most 8 x K) is re-read from
// cache. Coalesced when B and C have unit column stride.
template <typename R>
__global__ void __launch_bounds__(256) zgemm_smallm_kernel(GemmDesc d, const typename cvec<R>::T *__restrict__ A,
                                                           const typename cvec<R>::T *__restrict__ B,
                                                           typename cvec<R>::T *__restrict__ C) {
    typedef typename cvec<R>::T T;
    constexpr int MM = 8;
    const i64 total = (i64)d.batch * d.N;
    const bool use_beta = (d.beta.x != 0.0 || d.beta.y != 0.0);
    for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (i64)gridDim.x * blockDim.x) {
        const int b = (int)(t / d.N), n = (int)(t - (i64)b * d.N);
        T acc[MM];
#pragma unroll
        for (int m = 0; m < MM; ++m) acc[m] = cz<T>();
        for (int r = 0; r < d.nred; ++r) {
            const T *Ab = A + d.offA[(i64)b * d.nred + r];
            const T *Bb = B + d.offB[(i64)b * d.nred + r] + (i64)n * d.csB;
            for (int k = 0; k < d.K; ++k) {
                const T bv = Bb[(i64)k * d.rsB];
#pragma unroll
                for (int m = 0; m < MM; ++m)
                    if (m < d.M) cfma<T, R>(acc[m], Ab[(i64)m * d.rsA + (i64)k * d.csA], bv);
            }
        }
        T *Cb = C + d.offC[b] + (i64)n * d.csC;
#pragma unroll
        for (int m = 0; m < MM; ++m) {
            if (m >= d.M) break;
            T *c = Cb + (i64)m * d.rsC;
            T v;
            v.x = (R)d.alpha.x * acc[m].x - (R)d.alpha.y * acc[m].y;
            v.y = (R)d.alpha.x * acc[m].y + (R)d.alpha.y * acc[m].x;
            if (use_beta) {
                const T o = *c;
                v.x += (R)d.beta.x * o.x - (R)d.beta.y * o.y;
                v.y += (R)d.beta.x * o.y + (R)d.beta.y * o.x;
            }
            *c = v;
        }
    }
}

bool zgemm_smallm_supported(const GemmDesc &d) {
    return d.M >= 1 && d.M <= 8 && d.N >= 1 && d.batch >= 1 && (i64)d.K * d.nred <= 256;
}

template <typename R>
int launch_zgemm_smallm(const GemmDesc &d, const typename cvec<R>::T *A, const typename cvec<R>::T *B,
                        typename cvec<R>::T *C, cudaStream_t st) {
    if (!zgemm_smallm_supported(d)) return 0;
    const i64 g = ceil_div((i64)d.batch * d.N, 256);
    zgemm_smallm_kernel<R><<<(unsigned)(g > 152 * 16 ? 152 * 16 : g), 256, 0, st>>>(d, A, B, C);
    return 1;
}
template int launch_zgemm_smallm<double>(const GemmDesc &, const double2 *, const double2 *, double2 *, cudaStream_t);
template int launch_zgemm_smallm<float>(const GemmDesc &, const float2 *, const float2 *, float2 *, cudaStream_t);
template int launch_zgemm<double>(const GemmDesc &, const double2 *, const double2 *, double2 *, cudaStream_t, double2 *, i64);
template int launch_zgemm<float>(const GemmDesc &, const float2 *, const float2 *, float2 *, cudaStream_t, float2 *, i64);

// ----------------------------------------------------------------------------- batched permute-add
template <typename R>
__global__ void zpermute_kernel(PermDesc d, const typename cvec<R>::T *__restrict__ A, typename cvec<R>::T *C) {
    typedef typename cvec<R>::T T;
    const bool use_beta = (d.beta.x != 0.0 || d.beta.y != 0.0);
    for (int b = blockIdx.y; b < d.batch; b += gridDim.y) {
        const i64 oa0 = d.offA[b], oc0 = d.offC[b];
        for (i64 idx = (i64)blockIdx.x * blockDim.x + threadIdx.x; idx < d.total; idx += (i64)gridDim.x * blockDim.x) {
            i64 rem = idx, oa = oa0, oc = oc0;
            for (int dd = d.nd - 1; dd >= 0; --dd) {
                i64 q = rem / d.dims[dd];
                i64 id = rem - q * d.dims[dd];
                rem = q;
                oa += id * d.sA[dd];
                oc += id * d.sC[dd];
            }
            T a = A[oa];
            T v;
            v.x = (R)d.alpha.x * a.x - (R)d.alpha.y * a.y;
            v.y = (R)d.alpha.x * a.y + (R)d.alpha.y * a.x;
            if (use_beta) {
                T c = C[oc];
                v.x += (R)d.beta.x * c.x - (R)d.beta.y * c.y;
                v.y += (R)d.beta.x * c.y + (R)d.beta.y * c.x;
            }
            C[oc] = v;
        }
    }
}

template <typename R>
int launch_zpermute(const PermDesc &d, const typename cvec<R>::T *A, typename cvec<R>::T *C, cudaStream_t st) {
    if (d.batch <= 0 || d.total <= 0) return 0;
    i64 gx = ceil_div(d.total, 256);
    if (gx > 4096) gx = 4096;
    dim3 grid((unsigned)gx, (unsigned)(d.batch < 65535 ? d.batch : 65535));
    zpermute_kernel<R><<<grid, 256, 0, st>>>(d, A, C);
    return 1;
}
template int launch_zpermute<double>(const PermDesc &, const double2 *, double2 *, cudaStream_t);
template int launch_zpermute<float>(const PermDesc &, const float2 *, float2 *, cudaStream_t);

// ----------------------------------------------------------------------------- ABI <-> internal layout
// x: [nvec][D] (ABI), xt: [D][nv] (internal, columns >= nvec zero-filled)
__global__ void transpose_in_kernel(const double2 *__restrict__ x, double2 *__restrict__ xt, i64 D, int nvec, int nv) {
    __shared__ double2 tile[32][33];
    i64 d0 = (i64)blockIdx.x * 32;
    int v0 = blockIdx.y * 32;
    int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        int vv = v0 + r;
        i64 dd = d0 + tx;
        tile[r][tx] = (vv < nvec && dd < D) ? x[(i64)vv * D + dd] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        i64 dd = d0 + r;
        int vv = v0 + tx;
        if (dd < D && vv < nv) xt[dd * nv + vv] = tile[tx][r];
    }
}
__global__ void transpose_out_kernel(const double2 *__restrict__ yt, double2 *__restrict__ y, i64 D, int nvec, int nv) {
    __shared__ double2 tile[32][33];
    i64 d0 = (i64)blockIdx.x * 32;
    int v0 = blockIdx.y * 32;
    int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += 8) {
        i64 dd = d0 + r;
        int vv = v0 + tx;
        tile[r][tx] = (dd < D && vv < nv) ? yt[dd * nv + vv] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        int vv = v0 + r;
        i64 dd = d0 + tx;
        if (vv < nvec && dd < D) y[(i64)vv * D + dd] = tile[tx][r];
    }
}
void launch_transpose_in(const double2 *x, double2 *xt, i64 D, int nvec, int nv, cudaStream_t st) {
    dim3 grid((unsigned)ceil_div(D, 32), (unsigned)ceil_div(nv, 32));
    transpose_in_kernel<<<grid, dim3(32, 8), 0, st>>>(x, xt, D, nvec, nv);
}
void launch_transpose_out(const double2 *yt, double2 *y, i64 D, int nvec, int nv, cudaStream_t st) {
    dim3 grid((unsigned)ceil_div(D, 32), (unsigned)ceil_div(nv, 32));
    transpose_out_kernel<<<grid, dim3(32, 8), 0, st>>>(yt, y, D, nvec, nv);
}
