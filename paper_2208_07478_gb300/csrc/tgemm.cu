// Batched complex GEMM over tensor operands whose row, column and contraction indices are each a
// pair of tensor indices: index i of a GEMM dimension lives at (i / d2) * s1 + (i % d2) * s2 of
// its operand (IMap). A contraction such as sum_{n,f} W[(m,e),(n,f)] t[(n,f),(j,x)] over
// momentum-blocked tensors then runs as one launch, whatever the operands' index order, with no
// transposed copies: the build of the similarity-transformed Hamiltonian blocks (Eq. 5) and the
// sigma terms evaluated from the density-fitting factors use it.
//
// Tile: 64 x 64 complex outputs per CTA, 256 threads with 4 x 4 outputs each, 16 contraction
// indices staged through shared memory per step. Each thread's row / column offsets are computed
// once per tile; its contraction index is kept as (i / d2, i % d2) and advanced by 16 per step with
// two additions and a compare (no division in the loop: in FP32 the index arithmetic would
// otherwise cost as much as the multiply-adds).
#include "ccgf_internal.h"
#include <algorithm>

namespace {

constexpr int TB = 64, TK = 16;

__device__ __forceinline__ i64 imap(const IMap &m, i64 i) { return (i / m.d2) * m.s1 + (i % m.d2) * m.s2; }

// contraction index k < 2^31 of an IMap as (q, r) = (k / d2, k % d2), advanced by TK per step
struct KPos {
    int q, r;
};
__device__ __forceinline__ KPos kpos(const IMap &m, int k) {
    const int q = k / m.d2;
    return KPos{q, k - q * m.d2};
}
__device__ __forceinline__ void kadvance(const IMap &m, int q16, int r16, KPos &p) {
    p.r += r16;
    p.q += q16;
    if (p.r >= m.d2) {
        p.r -= m.d2;
        ++p.q;
    }
}
__device__ __forceinline__ i64 koff(const IMap &m, const KPos &p) { return (i64)p.q * m.s1 + (i64)p.r * m.s2; }

template <typename T> __device__ __forceinline__ T zero2();
template <> __device__ __forceinline__ double2 zero2<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 zero2<float2>() { return make_float2(0.f, 0.f); }

__device__ __forceinline__ double2 cvt2(double2 a, double2) { return a; }
__device__ __forceinline__ float2 cvt2(float2 a, float2) { return a; }
__device__ __forceinline__ float2 cvt2(double2 a, float2) { return make_float2((float)a.x, (float)a.y); }

// TA: storage type of A (double2 with R = float: an FP64 operand rounded to FP32 as it is loaded)
// ksplit > 1: grid z covers (batch, split); split s sums the reductions r in [s * rchunk, ...) (nred > 1)
// or the contraction range [s * kchunk, ...) (nred = 1) and writes raw partial sums to
// work[b][s][M][N]; tgemm_reduce_kernel applies alpha and beta.
template <typename R, typename TA>
__global__ void __launch_bounds__(256) tgemm_kernel(TGemm d, const TA *__restrict__ A, const typename cvec<R>::T *__restrict__ B,
                                                    typename cvec<R>::T *__restrict__ C, int ksplit, int kchunk,
                                                    typename cvec<R>::T *__restrict__ work) {
    typedef typename cvec<R>::T T;
    __shared__ T As[TK][TB + 1];
    __shared__ T Bs[TK][TB + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * TB, n0 = blockIdx.x * TB;
    // loader roles: A tile as 64 rows x 16 k (k fastest when the contraction index of A is
    // contiguous), B tile as 16 k x 64 columns (column fastest unless B's k index is contiguous)
    const bool a_kfast = d.ak.s2 == 1 && d.ak.d2 >= TK;
    const bool b_kfast = d.bk.s2 == 1 && d.bk.d2 >= TK && d.bn.s2 != 1;
    int a_row[4], a_kk[4], b_col[4], b_kk[4];
    i64 a_roff[4], b_coff[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int l = tid + 256 * s;
        if (a_kfast) { a_kk[s] = l & 15; a_row[s] = l >> 4; } else { a_row[s] = l & 63; a_kk[s] = l >> 6; }
        if (b_kfast) { b_kk[s] = l & 15; b_col[s] = l >> 4; } else { b_col[s] = l & 63; b_kk[s] = l >> 6; }
        const int m = m0 + a_row[s], n = n0 + b_col[s];
        a_roff[s] = m < d.M ? imap(d.am, m) : -1;
        b_coff[s] = n < d.N ? imap(d.bn, n) : -1;
    }
    const bool use_beta = d.beta.x != 0.0 || d.beta.y != 0.0;
    const int aq16 = TK / d.ak.d2, ar16 = TK % d.ak.d2, bq16 = TK / d.bk.d2, br16 = TK % d.bk.d2;
    for (int bz = blockIdx.z; bz < d.batch * ksplit; bz += gridDim.z) {
        const int b = bz / ksplit, ks = bz % ksplit;
        const int rchunk = d.nred > 1 ? (d.nred + ksplit - 1) / ksplit : 1;
        const int rbeg = d.nred > 1 ? ks * rchunk : 0, rend = d.nred > 1 ? min(d.nred, rbeg + rchunk) : 1;
        const int kbeg = d.nred > 1 ? 0 : ks * kchunk, kend = d.nred > 1 ? d.K : min(d.K, kbeg + kchunk);
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = zero2<T>();
        for (int r = rbeg; r < rend; ++r) {
            const TA *Ab = A + d.offA[(i64)b * d.nred + r];
            const T *Bb = B + d.offB[(i64)b * d.nred + r];
            KPos ap[4], bp[4];
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                ap[s] = kpos(d.ak, kbeg + a_kk[s]);
                bp[s] = kpos(d.bk, kbeg + b_kk[s]);
            }
            for (int k0 = kbeg; k0 < kend; k0 += TK) {
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    const int k = k0 + a_kk[s];
                    As[a_kk[s]][a_row[s]] = (a_roff[s] >= 0 && k < kend) ? cvt2(Ab[a_roff[s] + koff(d.ak, ap[s])], T()) : zero2<T>();
                    const int kb = k0 + b_kk[s];
                    Bs[b_kk[s]][b_col[s]] = (b_coff[s] >= 0 && kb < kend) ? Bb[koff(d.bk, bp[s]) + b_coff[s]] : zero2<T>();
                    kadvance(d.ak, aq16, ar16, ap[s]);
                    kadvance(d.bk, bq16, br16, bp[s]);
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < TK; ++kk) {
                    T a[4], bb[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                    for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            acc[i][j].x = fma(a[i].x, bb[j].x, acc[i][j].x);
                            acc[i][j].x = fma(-a[i].y, bb[j].y, acc[i][j].x);
                            acc[i][j].y = fma(a[i].x, bb[j].y, acc[i][j].y);
                            acc[i][j].y = fma(a[i].y, bb[j].x, acc[i][j].y);
                        }
                }
                __syncthreads();
            }
        }
        if (ksplit > 1) {
            T *Wb = work + ((i64)b * ksplit + ks) * (i64)d.M * d.N;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int m = m0 + ty + 16 * i;
                if (m >= d.M) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int n = n0 + tx + 16 * j;
                    if (n < d.N) Wb[(i64)m * d.N + n] = acc[i][j];
                }
            }
            continue;
        }
        T *Cb = C + d.offC[b];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int m = m0 + ty + 16 * i;
            if (m >= d.M) continue;
            const i64 rm = imap(d.cm, m);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = n0 + tx + 16 * j;
                if (n >= d.N) continue;
                T *c = Cb + rm + imap(d.cn, n);
                T v;
                v.x = (R)d.alpha.x * acc[i][j].x - (R)d.alpha.y * acc[i][j].y;
                v.y = (R)d.alpha.x * acc[i][j].y + (R)d.alpha.y * acc[i][j].x;
                if (use_beta) {
                    const T o = *c;
                    v.x += (R)d.beta.x * o.x - (R)d.beta.y * o.y;
                    v.y += (R)d.beta.x * o.y + (R)d.beta.y * o.x;
                }
                *c = v;
            }
        }
    }
}

template <typename R>
__global__ void tgemm_reduce_kernel(TGemm d, int ksplit, const typename cvec<R>::T *__restrict__ work, typename cvec<R>::T *__restrict__ C) {
    typedef typename cvec<R>::T T;
    const i64 mn = (i64)d.M * d.N;
    const bool use_beta = d.beta.x != 0.0 || d.beta.y != 0.0;
    for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t < mn * d.batch; t += (i64)gridDim.x * blockDim.x) {
        const int b = (int)(t / mn);
        const i64 e = t - (i64)b * mn;
        const int m = (int)(e / d.N), n = (int)(e - (i64)m * d.N);
        R sx = 0, sy = 0;
        for (int s = 0; s < ksplit; ++s) {
            const T p = work[((i64)b * ksplit + s) * mn + e];
            sx += p.x;
            sy += p.y;
        }
        T *c = C + d.offC[b] + imap(d.cm, m) + imap(d.cn, n);
        T v;
        v.x = (R)d.alpha.x * sx - (R)d.alpha.y * sy;
        v.y = (R)d.alpha.x * sy + (R)d.alpha.y * sx;
        if (use_beta) {
            const T o = *c;
            v.x += (R)d.beta.x * o.x - (R)d.beta.y * o.y;
            v.y += (R)d.beta.x * o.y + (R)d.beta.y * o.x;
        }
        *c = v;
    }
}

}  // namespace

// splits for a tensor GEMM whose output tiles cannot fill the GPU: enough (batch, split) blocks for two
// waves, each keeping at least 64 contraction steps of work (1: no split)
int tgemm_ksplit(const TGemm &d) {
    const i64 tiles = ceil_div(d.M, TB) * ceil_div(d.N, TB) * (i64)d.batch;
    if (tiles >= 304) return 1;
    const i64 work = (i64)d.K * d.nred;
    i64 s = ceil_div(304, tiles);
    s = std::min<i64>(s, std::max<i64>(1, work / 1024));
    if (d.nred > 1) s = std::min<i64>(s, d.nred);
    else s = std::min<i64>(s, std::max<i64>(1, d.K / 64));
    return (int)std::max<i64>(1, std::min<i64>(s, 64));
}
i64 tgemm_workspace_elems(const TGemm &d) {
    const int s = tgemm_ksplit(d);
    return s > 1 ? (i64)s * d.M * d.N * d.batch : 0;
}

IMap imap_single(i64 stride) { return IMap{1 << 30, 0, stride}; }
IMap imap_pair(int inner, i64 outer_stride, i64 inner_stride) { return IMap{inner, outer_stride, inner_stride}; }

template <typename R, typename TA>
static int launch_t(const TGemm &d, const TA *A, const typename cvec<R>::T *B, typename cvec<R>::T *C, cudaStream_t st,
                    typename cvec<R>::T *work, i64 work_elems) {
    if (d.batch <= 0 || d.M <= 0 || d.N <= 0 || d.nred <= 0) return 0;
    int ks = tgemm_ksplit(d);
    if (ks > 1 && (!work || work_elems < tgemm_workspace_elems(d))) ks = 1;
    int kchunk = d.K;
    if (ks > 1 && d.nred == 1) {
        kchunk = (int)(ceil_div(ceil_div(d.K, ks), TK) * TK);
        ks = (int)ceil_div(d.K, kchunk);
    } else if (ks > 1) {
        ks = (int)ceil_div(d.nred, ceil_div(d.nred, ks));   // every split non-empty
    }
    const i64 zt = (i64)d.batch * ks, z = zt < 65535 ? zt : 65535;
    dim3 grid((unsigned)ceil_div(d.N, TB), (unsigned)ceil_div(d.M, TB), (unsigned)z);
    tgemm_kernel<R, TA><<<grid, 256, 0, st>>>(d, A, B, C, ks, kchunk, work);
    if (ks == 1) return 1;
    const i64 n = (i64)d.M * d.N * d.batch, g = ceil_div(n, 256);
    tgemm_reduce_kernel<R><<<(unsigned)(g > 4096 ? 4096 : g), 256, 0, st>>>(d, ks, work, C);
    return 2;
}
template <typename R>
int launch_tgemm(const TGemm &d, const typename cvec<R>::T *A, const typename cvec<R>::T *B, typename cvec<R>::T *C,
                 cudaStream_t st, typename cvec<R>::T *work, i64 work_elems) {
    return launch_t<R, typename cvec<R>::T>(d, A, B, C, st, work, work_elems);
}
template int launch_tgemm<double>(const TGemm &, const double2 *, const double2 *, double2 *, cudaStream_t, double2 *, i64);
template int launch_tgemm<float>(const TGemm &, const float2 *, const float2 *, float2 *, cudaStream_t, float2 *, i64);
int launch_tgemm_a64(const TGemm &d, const double2 *A, const float2 *B, float2 *C, cudaStream_t st, float2 *work, i64 work_elems) {
    return launch_t<float, double2>(d, A, B, C, st, work, work_elems);
}

// a plain GemmDesc (single-stride indices) as a tensor GEMM
TGemm tgemm_of(const GemmDesc &g) {
    TGemm t{};
    t.M = g.M;
    t.N = g.N;
    t.K = g.K;
    t.nred = g.nred;
    t.batch = g.batch;
    t.am = imap_single(g.rsA);
    t.ak = imap_single(g.csA);
    t.bk = imap_single(g.rsB);
    t.bn = imap_single(g.csB);
    t.cm = imap_single(g.rsC);
    t.cn = imap_single(g.csC);
    t.offA = g.offA;
    t.offB = g.offB;
    t.offC = g.offC;
    t.alpha = g.alpha;
    t.beta = g.beta;
    return t;
}
