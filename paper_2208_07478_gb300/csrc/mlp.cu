// Learned warm start for the shifted GMRES solves: a per-element MLP that predicts the
// initial vector of a right-hand side (sector, K, orbital p, frequency w) from the converged
// solutions of the same right-hand side at the two nearest solved training frequencies.
//
// Features of element mu of column (p, w), with w- <= w <= w+ the neighbouring training
// frequencies, x-/x+ their solutions, d the one-body diagonal of A, z(w) = w -+ i eta,
// s = +1 (IP) / -1 (EA), g(w') = 1 / (z(w') + s d_mu), and the baseline
//   base = (1 - t) x- g(w)/g(w-) + t x+ g(w)/g(w+),   t = (w - w-) / (w+ - w-)
// (the neighbours carried to w along the element's own diagonal resolvent):
//   eta x- / |b_p|, eta x+ / |b_p|, eta base / |b_p| (re, im each), t, (w+ - w-) / (10 eta),
//   eta g(w), eta g(w-), eta g(w+) (re, im each)                                  -> F = 14.
// Output: the correction eta (x0 - base) / |b_p| (re, im) divided by (span / (10 eta))^2, span =
// w+ - w-: the error of an interpolation between neighbours grows with the square of their
// spacing, so this scaling carries what is learned on training triples (neighbours two grid
// steps apart) to inference between adjacent points. The last layer starts at zero, so an
// untrained network predicts the baseline. Network: tanh(f W1 + b1) -> tanh(. W2 + b2) -> . W3 + b3,
// hidden 256; FP32 master weights, forward with bfloat16-rounded weight matrices, FP32
// accumulation. Training: Adam on the mean squared error against converged solutions at
// interior training frequencies (each one predicted from neighbours one or two grid steps away).
#include "ccgf_internal.h"
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <random>

namespace {

constexpr int kF = 14;
constexpr int kH = 256;

// ----------------------------------------------------------------------------- real FP32 GEMM
// C[m,n] = act(alpha * sum_k A[m,k] B[k,n] + beta C[m,n] + bias[n]), 64x64 tiles, 4x4 per thread.
// ksplit > 1: K is split over gridDim.z and partial sums are added atomically (C pre-zeroed,
// alpha only, no bias/act/beta) - used for the weight gradients (long K = rows).
struct SG {
    int M, N, K;
    i64 rsA, csA, rsB, csB, rsC, csC;
    float alpha, beta;
    const float *bias;
    int act;      // 0 none, 1 tanh
    int ksplit;
};

__global__ void __launch_bounds__(256) sgemm_kernel(SG d, const float *__restrict__ A, const float *__restrict__ B, float *C) {
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int kchunk = (d.K + d.ksplit - 1) / d.ksplit;
    const int kbeg = blockIdx.z * kchunk, kend = min(d.K, kbeg + kchunk);
    float acc[4][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += 16) {
        for (int s = 0; s < 4; ++s) {
            int l = tid + 256 * s, i, kk;
            if (d.csA == 1) { kk = l & 15; i = l >> 4; } else { i = l & 63; kk = l >> 6; }
            int m = m0 + i, k = k0 + kk;
            As[kk][i] = (m < d.M && k < kend) ? A[(i64)m * d.rsA + (i64)k * d.csA] : 0.f;
        }
        for (int s = 0; s < 4; ++s) {
            int l = tid + 256 * s, nn, kk;
            if (d.csB == 1) { nn = l & 63; kk = l >> 6; } else { kk = l & 15; nn = l >> 4; }
            int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < d.N && k < kend) ? B[(i64)k * d.rsB + (i64)n * d.csB] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = m0 + ty + 16 * i;
        if (m >= d.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + tx + 16 * j;
            if (n >= d.N) continue;
            float *c = C + (i64)m * d.rsC + (i64)n * d.csC;
            if (d.ksplit > 1) {
                atomicAdd(c, d.alpha * acc[i][j]);
                continue;
            }
            float v = d.alpha * acc[i][j];
            if (d.beta != 0.f) v += d.beta * *c;
            if (d.bias) v += d.bias[n];
            if (d.act == 1) v = tanhf(v);
            *c = v;
        }
    }
}

int sgemm(const SG &d0, const float *A, const float *B, float *C, cudaStream_t st) {
    SG d = d0;
    if (d.ksplit < 1) d.ksplit = 1;
    dim3 grid((unsigned)ceil_div(d.N, 64), (unsigned)ceil_div(d.M, 64), (unsigned)d.ksplit);
    sgemm_kernel<<<grid, 256, 0, st>>>(d, A, B, C);
    return 1;
}
SG sg(int M, int N, int K, i64 rsA, i64 csA, i64 rsB, i64 csB, i64 rsC, float beta = 0.f, const float *bias = nullptr,
      int act = 0, int ksplit = 1) {
    SG d{};
    d.M = M; d.N = N; d.K = K;
    d.rsA = rsA; d.csA = csA; d.rsB = rsB; d.csB = csB; d.rsC = rsC; d.csC = 1;
    d.alpha = 1.f; d.beta = beta; d.bias = bias; d.act = act; d.ksplit = ksplit;
    return d;
}

__global__ void round_bf16_kernel(const float *a, float *b, i64 n) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
        b[i] = __bfloat162float(__float2bfloat16_rn(a[i]));
}
// dy = 2 (y - t) / n, loss += sum (y - t)^2 / n
__global__ void loss_grad_kernel(const float *y, const float *t, float *dy, i64 n2, double inv_n, double *loss) {
    double acc = 0;
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (i64)gridDim.x * blockDim.x) {
        float r = y[i] - t[i];
        dy[i] = (float)(2.0 * r * inv_n);
        acc += (double)r * r * inv_n;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}
// g *= 1 - h^2
__global__ void tanh_back_kernel(float *g, const float *h, i64 n) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) g[i] *= 1.f - h[i] * h[i];
}
// out[j] = sum_r a[r][j]   (out zeroed; rows strided over blocks)
__global__ void colsum_kernel(const float *a, i64 rows, int cols, float *out) {
    for (int j = threadIdx.x; j < cols; j += blockDim.x) {
        float acc = 0.f;
        for (i64 r = blockIdx.x; r < rows; r += gridDim.x) acc += a[r * cols + j];
        atomicAdd(out + j, acc);
    }
}
__global__ void adam_kernel(float *th, float *m, float *v, const float *g, i64 n, float lr, float b1, float b2, float c1, float c2) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.f - b1) * gi;
        float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        th[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    }
}

// Fm = (Fm - mean) / std per feature; T /= tscale (when T is given)
__global__ void normalize_kernel(float *Fm, i64 rows, int F, const float *mean, const float *inv_std, float *T, float inv_t) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < rows * F; i += (i64)gridDim.x * blockDim.x) {
        int f = i % F;
        Fm[i] = (Fm[i] - mean[f]) * inv_std[f];
    }
    if (T)
        for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < rows * 2; i += (i64)gridDim.x * blockDim.x) T[i] *= inv_t;
}
// Y *= tscale
__global__ void scale_kernel(float *Y, i64 n, float s) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) Y[i] *= s;
}

inline unsigned gsz(i64 n) { return (unsigned)std::max<i64>(1, std::min<i64>(ceil_div(n, 256), 152 * 16)); }

// parameter offsets: W1 [F,H], b1 [H], W2 [H,H], b2 [H], W3 [H,2], b3 [2]
struct POff {
    i64 W1, b1, W2, b2, W3, b3, n;
};
POff poff(int F, int H) {
    POff p;
    p.W1 = 0;
    p.b1 = p.W1 + (i64)F * H;
    p.W2 = p.b1 + H;
    p.b2 = p.W2 + (i64)H * H;
    p.W3 = p.b2 + H;
    p.b3 = p.W3 + 2 * H;
    p.n = p.b3 + 2;
    return p;
}

// Forward on rows x F features; th: parameters used (already bf16-rounded when requested).
int forward(const float *th, int F, int H, i64 rows, const float *X, float *H1, float *H2, float *Y, cudaStream_t st) {
    POff o = poff(F, H);
    int n = 0;
    n += sgemm(sg((int)rows, H, F, F, 1, H, 1, H, 0.f, th + o.b1, 1), X, th + o.W1, H1, st);
    n += sgemm(sg((int)rows, H, H, H, 1, H, 1, H, 0.f, th + o.b2, 1), H1, th + o.W2, H2, st);
    n += sgemm(sg((int)rows, 2, H, H, 1, 2, 1, 2, 0.f, th + o.b3, 0), H2, th + o.W3, Y, st);
    return n;
}

// Loss and gradient (w.r.t. the parameters, through the rounded weights thr) on rows.
int backward(const float *thr, int F, int H, i64 rows, const float *X, const float *T, float *H1, float *H2, float *Y,
             float *dZ1, float *dZ2, float *grad, double *loss_dev, cudaStream_t st) {
    POff o = poff(F, H);
    int n = forward(thr, F, H, rows, X, H1, H2, Y, st);
    cudaMemsetAsync(grad, 0, sizeof(float) * o.n, st);
    loss_grad_kernel<<<gsz(rows * 2), 256, 0, st>>>(Y, T, Y, rows * 2, 1.0 / (double)rows, loss_dev);   // Y becomes dY
    n++;
    const int ks = (int)std::max<i64>(1, std::min<i64>(64, rows / 2048));
    // dW3 = H2^T dY, db3 = colsum dY
    n += sgemm(sg(H, 2, (int)rows, 1, H, 2, 1, 2, 0.f, nullptr, 0, ks), H2, Y, grad + o.W3, st);
    colsum_kernel<<<64, 32, 0, st>>>(Y, rows, 2, grad + o.b3);
    n++;
    // dZ2 = (dY W3^T) * (1 - H2^2)
    n += sgemm(sg((int)rows, H, 2, 2, 1, 1, 2, H), Y, thr + o.W3, dZ2, st);
    tanh_back_kernel<<<gsz(rows * H), 256, 0, st>>>(dZ2, H2, rows * H);
    n++;
    n += sgemm(sg(H, H, (int)rows, 1, H, H, 1, H, 0.f, nullptr, 0, ks), H1, dZ2, grad + o.W2, st);
    colsum_kernel<<<128, 256, 0, st>>>(dZ2, rows, H, grad + o.b2);
    n++;
    // dZ1 = (dZ2 W2^T) * (1 - H1^2)
    n += sgemm(sg((int)rows, H, H, H, 1, 1, H, H), dZ2, thr + o.W2, dZ1, st);
    tanh_back_kernel<<<gsz(rows * H), 256, 0, st>>>(dZ1, H1, rows * H);
    n++;
    n += sgemm(sg(F, H, (int)rows, 1, F, H, 1, H, 0.f, nullptr, 0, ks), X, dZ1, grad + o.W1, st);
    colsum_kernel<<<128, 256, 0, st>>>(dZ1, rows, H, grad + o.b1);
    n++;
    return n;
}

// rounded copy of the weight matrices (biases copied as they are)
int round_params(const float *th, float *thr, int F, int H, int bf16, cudaStream_t st) {
    POff o = poff(F, H);
    cudaMemcpyAsync(thr, th, sizeof(float) * o.n, cudaMemcpyDeviceToDevice, st);
    if (!bf16) return 0;
    round_bf16_kernel<<<gsz(o.b1), 256, 0, st>>>(th + o.W1, thr + o.W1, (i64)F * H);
    round_bf16_kernel<<<gsz((i64)H * H), 256, 0, st>>>(th + o.W2, thr + o.W2, (i64)H * H);
    round_bf16_kernel<<<gsz(2 * H), 256, 0, st>>>(th + o.W3, thr + o.W3, 2 * (i64)H);
    return 3;
}

// ----------------------------------------------------------------------------- features
struct FeatArgs {
    i64 D;                    // full dimension (stride of a training slab)
    i64 mu0, nmu;             // element rows handled by this launch
    int N, nv, nw;
    double eta, s;
    const double *d;          // [D] diagonal estimate
    const double *bnorm;      // [N] |b_p|
    const int *wlo, *whi;     // [nw] training index of the neighbours
    const double *om;         // [nw] target frequencies
    const double *tom;        // training frequencies
    const double2 *store;     // [n_train][D][N]
};
__device__ __forceinline__ void feat_row(const FeatArgs &a, i64 mu, int p, int w, float *f, double2 *base_out) {
    const int il = a.wlo[w], ih = a.whi[w];
    const double wl = a.tom[il], wh = a.tom[ih], om = a.om[w];
    const double2 xl = a.store[((i64)il * a.D + mu) * a.N + p];
    const double2 xh = a.store[((i64)ih * a.D + mu) * a.N + p];
    const double sc = a.eta / (a.bnorm[p] > 0 ? a.bnorm[p] : 1.0);
    const double zi = a.s > 0 ? -a.eta : a.eta;   // Im z
    const double dd = a.s * a.d[mu];
    // q(w') = z(w') + s d: g = 1/q; ratio g(w)/g(w') = q(w')/q(w)
    auto ratio = [&](double w_) -> double2 {
        double nr = w_ + dd, ni = zi, drr = om + dd, dri = zi;
        double den = drr * drr + dri * dri;
        return make_double2((nr * drr + ni * dri) / den, (ni * drr - nr * dri) / den);
    };
    auto cmulx = [](double2 a_, double2 b_) { return make_double2(a_.x * b_.x - a_.y * b_.y, a_.x * b_.y + a_.y * b_.x); };
    const double span = wh - wl;
    const double t = span > 0 ? (om - wl) / span : 0.5;
    const double2 bl = cmulx(xl, ratio(wl)), bh = cmulx(xh, ratio(wh));
    const double2 base = make_double2((1 - t) * bl.x + t * bh.x, (1 - t) * bl.y + t * bh.y);
    auto g = [&](double w_, float *o2) {
        double re = w_ + dd, im = zi;
        double den = re * re + im * im;
        o2[0] = (float)(a.eta * re / den);
        o2[1] = (float)(-a.eta * im / den);
    };
    f[0] = (float)(sc * xl.x);
    f[1] = (float)(sc * xl.y);
    f[2] = (float)(sc * xh.x);
    f[3] = (float)(sc * xh.y);
    f[4] = (float)(sc * base.x);
    f[5] = (float)(sc * base.y);
    f[6] = (float)t;
    f[7] = (float)(span / (10.0 * a.eta));
    g(om, f + 8);
    g(wl, f + 10);
    g(wh, f + 12);
    *base_out = base;
}
// inference rows r = (mu - mu0) * nv + c, c = p * nw + w
__global__ void features_kernel(FeatArgs a, float *Fm, double2 *Base) {
    const i64 rows = a.nmu * a.nv;
    for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (i64)gridDim.x * blockDim.x) {
        const i64 mu = a.mu0 + r / a.nv;
        const int c = r % a.nv, p = c / a.nw, w = c % a.nw;
        feat_row(a, mu, p, w, Fm + r * kF, Base + r);
    }
}
// x0[mu][c] = base + (y0 + i y1) |b_p| / eta for rows of the chunk starting at element mu0
__global__ void apply_kernel(const float *Y, const double2 *Base, const double *bnorm, const double *span2, double eta, i64 mu0,
                             i64 nmu, int nv, int nw, double2 *X, double2 *Xbase) {
    const i64 rows = nmu * nv;
    for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (i64)gridDim.x * blockDim.x) {
        const int c = r % nv, p = c / nw;
        const double sc = bnorm[p] / eta * span2[c % nw];
        X[mu0 * nv + r] = make_double2(Base[r].x + sc * Y[2 * r], Base[r].y + sc * Y[2 * r + 1]);
        if (Xbase) Xbase[mu0 * nv + r] = Base[r];
    }
}
__device__ __forceinline__ unsigned hash32(unsigned x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}
// training rows mixed over k-points and interior training frequencies of one sector:
// row r draws (K, i, mu, p); store_all [nk][n][D][N], d_all [nk][D], bnorm_all [nk][N]
__global__ void train_rows_mixed_kernel(FeatArgs a, int nk, int n, const double2 *store_all, const double *d_all,
                                        const double *bnorm_all, unsigned seed, i64 rows, float *Fm, float *T) {
    for (i64 r = (i64)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (i64)gridDim.x * blockDim.x) {
        unsigned h1 = hash32(seed ^ (unsigned)(r * 2654435761u)), h2 = hash32(h1 + 0x9e3779b9u), h3 = hash32(h2 + 0x7f4a7c15u);
        const int K = (int)(((unsigned long long)h3 * (unsigned long long)nk) >> 32);
        const int i = 1 + (int)(((unsigned long long)hash32(h3 ^ 0x85ebca6bu) * (unsigned long long)(n - 2)) >> 32);
        const i64 mu = (i64)(((unsigned long long)h1 * (unsigned long long)a.D) >> 32);
        const int p = (int)(((unsigned long long)h2 * (unsigned long long)a.N) >> 32);
        FeatArgs b = a;
        b.store = store_all + (i64)K * n * a.D * a.N;
        b.d = d_all + (i64)K * a.D;
        b.bnorm = bnorm_all + (i64)K * a.N;
        // neighbours i - a, i + b of training point i, a, b in {1, 2} where the grid allows: varied
        // positions t and spans (w index 0 of per-row tables is not used)
        const unsigned h4 = hash32(h1 ^ 0xc2b2ae35u);
        const int a_off = (i >= 2 && (h4 & 1)) ? 2 : 1, b_off = (i + 2 <= n - 1 && (h4 & 2)) ? 2 : 1;
        const int il = i - a_off, ih = i + b_off;
        int lo_hi[2] = {il, ih};
        double om = a.tom[i];
        b.wlo = lo_hi;
        b.whi = lo_hi + 1;
        b.om = &om;
        double2 base;
        feat_row(b, mu, p, 0, Fm + r * kF, &base);
        const double2 x = b.store[((i64)i * a.D + mu) * a.N + p];
        const double sf = (a.tom[ih] - a.tom[il]) / (10.0 * a.eta);
        const double sc = a.eta / (b.bnorm[p] > 0 ? b.bnorm[p] : 1.0) / (sf * sf);
        T[2 * r] = (float)(sc * (x.x - base.x));
        T[2 * r + 1] = (float)(sc * (x.y - base.y));
    }
}

}  // namespace

// ----------------------------------------------------------------------------- state
struct WarmStart {
    int F = kF, H = kH, bf16 = 1;
    bool trained = false;
    double eta = 0;
    std::vector<double> omega;            // training frequencies (ascending)
    DBuf<double2> store[2];               // per sector: [nk][n_train][D][N]
    DBuf<double> bnorm[2];                // per sector: [nk][N]
    DBuf<double> tom;                     // training frequencies on device
    DBuf<float> th, thr, m, v, grad;
    DBuf<float> Fm, H1, H2, Y, T, dZ1, dZ2;
    DBuf<double2> Base;
    DBuf<double> loss;
    i64 rows_cap = 0;
    i64 steps = 0;
    double val_net = 0, val_base = 0;   // validation losses: network, baseline alone
    bool use_net = false;
    DBuf<float> fmean, finv;            // feature standardisation
    float tscale = 1.f;                 // target scale (network outputs are multiplied by it)
};

void warmstart_free(ccgf_handle *h) {
    WarmStart *w = h->ws;
    if (!w) return;
    for (int s = 0; s < 2; ++s) {
        dfree(w->store[s]);
        dfree(w->bnorm[s]);
    }
    DBuf<float> *fb[] = {&w->th, &w->thr, &w->m, &w->v, &w->grad, &w->Fm, &w->H1, &w->H2, &w->Y, &w->T, &w->dZ1, &w->dZ2};
    for (auto *b : fb) dfree(*b);
    dfree(w->tom);
    dfree(w->loss);
    dfree(w->Base);
    dfree(w->fmean);
    dfree(w->finv);
    delete w;
    h->ws = nullptr;
}

static ccgf_status ensure_rows(WarmStart *w, i64 rows) {
    if (rows <= w->rows_cap) return CCGF_OK;
    DBuf<float> *fb[] = {&w->Fm, &w->H1, &w->H2, &w->Y, &w->T, &w->dZ1, &w->dZ2};
    for (auto *b : fb) dfree(*b);
    dfree(w->Base);
    CCGF_TRY(dalloc(w->Base, rows));
    CCGF_TRY(dalloc(w->Fm, rows * w->F));
    CCGF_TRY(dalloc(w->H1, rows * w->H));
    CCGF_TRY(dalloc(w->H2, rows * w->H));
    CCGF_TRY(dalloc(w->Y, rows * 2));
    CCGF_TRY(dalloc(w->T, rows * 2));
    CCGF_TRY(dalloc(w->dZ1, rows * w->H));
    CCGF_TRY(dalloc(w->dZ2, rows * w->H));
    w->rows_cap = rows;
    return CCGF_OK;
}

// Storage of training solutions, filled by the solver while it runs the training grid.
ccgf_status warmstart_begin_capture(ccgf_handle *h, const double *omega, int n, double eta) {
    warmstart_free(h);
    WarmStart *w = new WarmStart();
    h->ws = w;
    w->omega.assign(omega, omega + n);
    w->eta = eta;
    CCGF_TRY(dalloc(w->tom, n));
    CCGF_CUDA_TRY(cudaMemcpy(w->tom.p, omega, sizeof(double) * n, cudaMemcpyHostToDevice));
    for (int s = 0; s < 2; ++s) {
        const i64 D = s == 0 ? h->dim_ip : h->dim_ea;
        CCGF_TRY(dalloc(w->store[s], (i64)h->nk * n * D * h->n));
        CCGF_TRY(dalloc(w->bnorm[s], (i64)h->nk * h->n));
    }
    return CCGF_OK;
}

// Called by the solver after each batch when a capture is active: X [D][nv], c = p * nw + w.
__global__ void capture_kernel(const double2 *X, i64 D, int N, int nw, int w0, int ntrain, double2 *store_k) {
    const int nv = N * nw;
    for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t < D * nv; t += (i64)gridDim.x * blockDim.x) {
        const i64 mu = t / nv;
        const int c = t % nv, p = c / nw, w = c % nw;
        if (w0 + w < ntrain) store_k[((i64)(w0 + w) * D + mu) * N + p] = X[t];
    }
}
ccgf_status warmstart_capture(ccgf_handle *h, int sector, int K, const double2 *X, i64 D, int nw, int w0, const double *bnorm2_h,
                              cudaStream_t st) {
    WarmStart *w = h->ws;
    if (!w) return CCGF_OK;
    const int si = sector - 1, n = (int)w->omega.size(), N = h->n;
    double2 *store_k = w->store[si].p + (i64)K * n * D * N;
    capture_kernel<<<gsz(D * N * nw), 256, 0, st>>>(X, D, N, nw, w0, n, store_k);
    h->launches++;
    std::vector<double> bn(N);
    for (int p = 0; p < N; ++p) bn[p] = std::sqrt(bnorm2_h[p * nw]);
    CCGF_CUDA_TRY(cudaMemcpyAsync(w->bnorm[si].p + (i64)K * N, bn.data(), sizeof(double) * N, cudaMemcpyHostToDevice, st));
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    return CCGF_OK;
}

static void neighbours(const std::vector<double> &tw, const double *om, int nw, std::vector<int> &lo, std::vector<int> &hi) {
    const int n = (int)tw.size();
    lo.resize(nw);
    hi.resize(nw);
    for (int j = 0; j < nw; ++j) {
        // nearest training points below and above (the two end points outside the grid)
        int k = (int)(std::upper_bound(tw.begin(), tw.end(), om[j]) - tw.begin());
        k = std::min(std::max(k, 1), n - 1);
        lo[j] = k - 1;
        hi[j] = k;
    }
}

// Predict x0 for the columns c = p * nw + w of a batch at frequencies om[0..nw) (host array)
// into X [D][nv]. *used = false (X untouched) without a trained network.
ccgf_status warmstart_infer(ccgf_handle *h, int sector, int K, const double *om, int nw, const double *dvec, double2 *X,
                            double2 *Xbase, bool *used, bool *net, cudaStream_t st) {
    *used = false;
    *net = false;
    WarmStart *w = h->ws;
    if (!w || !w->trained || w->omega.size() < 2) return CCGF_OK;
    const int si = sector - 1, N = h->n, n = (int)w->omega.size();
    const i64 D = sector == CCGF_SECTOR_IP ? h->dim_ip : h->dim_ea;
    const int nv = N * nw;
    std::vector<int> lo, hi;
    neighbours(w->omega, om, nw, lo, hi);
    // (span / (10 eta))^2 per column frequency: the scale of the learned correction
    std::vector<double> span2(nw);
    for (int j = 0; j < nw; ++j) {
        const double sf = (w->omega[hi[j]] - w->omega[lo[j]]) / (10.0 * w->eta);
        span2[j] = sf * sf;
    }
    DBuf<int> dlo, dhi;
    DBuf<double> dom, dspan2;
    CCGF_TRY(dalloc(dlo, nw));
    CCGF_TRY(dalloc(dhi, nw));
    CCGF_TRY(dalloc(dom, nw));
    CCGF_TRY(dalloc(dspan2, nw));
    CCGF_CUDA_TRY(cudaMemcpyAsync(dlo.p, lo.data(), sizeof(int) * nw, cudaMemcpyHostToDevice, st));
    CCGF_CUDA_TRY(cudaMemcpyAsync(dhi.p, hi.data(), sizeof(int) * nw, cudaMemcpyHostToDevice, st));
    CCGF_CUDA_TRY(cudaMemcpyAsync(dom.p, om, sizeof(double) * nw, cudaMemcpyHostToDevice, st));
    CCGF_CUDA_TRY(cudaMemcpyAsync(dspan2.p, span2.data(), sizeof(double) * nw, cudaMemcpyHostToDevice, st));
    FeatArgs a{};
    a.D = D;
    a.N = N;
    a.nv = nv;
    a.nw = nw;
    a.eta = w->eta;
    a.s = sector == CCGF_SECTOR_IP ? 1.0 : -1.0;
    a.d = dvec;
    a.bnorm = w->bnorm[si].p + (i64)K * N;
    a.wlo = dlo.p;
    a.whi = dhi.p;
    a.om = dom.p;
    a.tom = w->tom.p;
    a.store = w->store[si].p + (i64)K * n * D * N;
    h->launches += round_params(w->th.p, w->thr.p, w->F, w->H, w->bf16, st);
    const i64 mu_chunk = std::max<i64>(1, (i64)(1 << 19) / nv);
    ccgf_status s = ensure_rows(w, mu_chunk * nv);
    if (s != CCGF_OK) { dfree(dlo); dfree(dhi); dfree(dom); dfree(dspan2); return s; }
    for (i64 mu0 = 0; mu0 < D; mu0 += mu_chunk) {
        a.mu0 = mu0;
        a.nmu = std::min(mu_chunk, D - mu0);
        const i64 rows = a.nmu * nv;
        features_kernel<<<gsz(rows), 256, 0, st>>>(a, w->Fm.p, w->Base.p);
        normalize_kernel<<<gsz(rows * w->F), 256, 0, st>>>(w->Fm.p, rows, w->F, w->fmean.p, w->finv.p, nullptr, 1.f);
        h->launches += 2 + forward(w->thr.p, w->F, w->H, rows, w->Fm.p, w->H1.p, w->H2.p, w->Y.p, st);
        scale_kernel<<<gsz(rows * 2), 256, 0, st>>>(w->Y.p, rows * 2, w->tscale);
        h->launches++;
        apply_kernel<<<gsz(rows), 256, 0, st>>>(w->Y.p, w->Base.p, a.bnorm, dspan2.p, w->eta, mu0, a.nmu, nv, nw, X,
                                                w->use_net ? Xbase : nullptr);
        h->launches++;
    }
    CCGF_CUDA_TRY(cudaGetLastError());
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(dlo);
    dfree(dhi);
    dfree(dom);
    dfree(dspan2);
    *used = true;
    *net = w->use_net;
    return CCGF_OK;
}

// Adam on random rows of interior training frequencies (each predicted from its neighbours).
ccgf_status warmstart_train(ccgf_handle *h, int sectors, int steps, i64 rows, double lr, unsigned seed, double *final_loss,
                            cudaStream_t st) {
    WarmStart *w = h->ws;
    const int n = (int)w->omega.size();
    if (n < 3) { set_last_error("the warm start needs at least 3 training frequencies"); return CCGF_ERR_INVALID_ARG; }
    if (steps < 0) { set_last_error("steps must be >= 0"); return CCGF_ERR_INVALID_ARG; }
    POff o = poff(w->F, w->H);
    CCGF_TRY(dalloc(w->th, o.n));
    CCGF_TRY(dalloc(w->thr, o.n));
    CCGF_TRY(dalloc(w->m, o.n));
    CCGF_TRY(dalloc(w->v, o.n));
    CCGF_TRY(dalloc(w->grad, o.n));
    CCGF_TRY(dalloc(w->loss, 1));
    CCGF_TRY(ensure_rows(w, rows));
    // Glorot-uniform weights, zero biases (host RNG, seeded)
    std::vector<float> th(o.n, 0.f);
    std::mt19937 gen(seed);
    auto fill = [&](i64 off, int fi, int fo) {
        float lim = std::sqrt(6.f / (fi + fo));
        std::uniform_real_distribution<float> U(-lim, lim);
        for (i64 k = 0; k < (i64)fi * fo; ++k) th[off + k] = U(gen);
    };
    fill(o.W1, w->F, w->H);
    fill(o.W2, w->H, w->H);   // W3, b3 stay zero: the untrained network predicts the baseline
    CCGF_CUDA_TRY(cudaMemcpyAsync(w->th.p, th.data(), sizeof(float) * o.n, cudaMemcpyHostToDevice, st));
    CCGF_CUDA_TRY(cudaMemsetAsync(w->m.p, 0, sizeof(float) * o.n, st));
    CCGF_CUDA_TRY(cudaMemsetAsync(w->v.p, 0, sizeof(float) * o.n, st));
    std::vector<int> secs;
    for (int sec = 1; sec <= 2; ++sec)
        if (sectors & sec) secs.push_back(sec);
    const float b1 = 0.9f, b2 = 0.999f;
    double last = 0;
    // diagonal estimates of every (sector, K), kept for the whole training
    DBuf<double> dall[2];
    for (int sec : secs) {
        const i64 D = sec == CCGF_SECTOR_IP ? h->dim_ip : h->dim_ea;
        CCGF_TRY(dalloc(dall[sec - 1], (i64)h->nk * D));
        for (int K = 0; K < h->nk; ++K) CCGF_TRY(diag_estimate_device(h, sec, K, dall[sec - 1].p + (i64)K * D, st));
    }
    // one mini-batch of training rows of a sector, mixed over k-points and interior frequencies
    auto make_batch = [&](int it, unsigned salt) -> ccgf_status {
        const int sec = secs[it % secs.size()];
        const i64 D = sec == CCGF_SECTOR_IP ? h->dim_ip : h->dim_ea;
        FeatArgs a{};
        a.D = D;
        a.N = h->n;
        a.nv = 1;
        a.nw = 1;
        a.eta = w->eta;
        a.s = sec == CCGF_SECTOR_IP ? 1.0 : -1.0;
        a.tom = w->tom.p;
        train_rows_mixed_kernel<<<gsz(rows), 256, 0, st>>>(a, h->nk, n, w->store[sec - 1].p, dall[sec - 1].p,
                                                           w->bnorm[sec - 1].p, seed * 7919u + (unsigned)it + salt, rows,
                                                           w->Fm.p, w->T.p);
        h->launches++;
        if (w->fmean.p) {
            normalize_kernel<<<gsz(rows * w->F), 256, 0, st>>>(w->Fm.p, rows, w->F, w->fmean.p, w->finv.p, w->T.p, 1.f / w->tscale);
            h->launches++;
        }
        return CCGF_OK;
    };
    // feature means / standard deviations and the target scale from a few raw batches
    {
        const int nstat = 4;
        std::vector<double> s1(w->F, 0.0), s2(w->F, 0.0);
        double t2 = 0;
        std::vector<float> fh(rows * w->F), th_(2 * rows);
        for (int k = 0; k < nstat; ++k) {
            CCGF_TRY(make_batch(k, 0x27d4eb2du));
            CCGF_CUDA_TRY(cudaMemcpyAsync(fh.data(), w->Fm.p, sizeof(float) * fh.size(), cudaMemcpyDeviceToHost, st));
            CCGF_CUDA_TRY(cudaMemcpyAsync(th_.data(), w->T.p, sizeof(float) * th_.size(), cudaMemcpyDeviceToHost, st));
            CCGF_CUDA_TRY(cudaStreamSynchronize(st));
            for (i64 r = 0; r < rows; ++r)
                for (int f = 0; f < w->F; ++f) {
                    double x = fh[r * w->F + f];
                    s1[f] += x;
                    s2[f] += x * x;
                }
            for (float x : th_) t2 += (double)x * x;
        }
        const double cnt = (double)nstat * rows;
        std::vector<float> mean(w->F), inv(w->F);
        for (int f = 0; f < w->F; ++f) {
            double mu = s1[f] / cnt, var = std::max(s2[f] / cnt - mu * mu, 0.0);
            mean[f] = (float)mu;
            inv[f] = (float)(var > 1e-30 ? 1.0 / std::sqrt(var) : 1.0);
        }
        w->tscale = (float)std::max(std::sqrt(t2 / (2.0 * cnt)), 1e-30);
        CCGF_TRY(dalloc(w->fmean, w->F));
        CCGF_TRY(dalloc(w->finv, w->F));
        CCGF_CUDA_TRY(cudaMemcpyAsync(w->fmean.p, mean.data(), sizeof(float) * w->F, cudaMemcpyHostToDevice, st));
        CCGF_CUDA_TRY(cudaMemcpyAsync(w->finv.p, inv.data(), sizeof(float) * w->F, cudaMemcpyHostToDevice, st));
    }
    for (int it = 0; it < steps; ++it) {
        CCGF_TRY(make_batch(it, 0u));
        h->launches += round_params(w->th.p, w->thr.p, w->F, w->H, w->bf16, st);
        CCGF_CUDA_TRY(cudaMemsetAsync(w->loss.p, 0, sizeof(double), st));
        h->launches += backward(w->thr.p, w->F, w->H, rows, w->Fm.p, w->T.p, w->H1.p, w->H2.p, w->Y.p, w->dZ1.p, w->dZ2.p,
                                w->grad.p, w->loss.p, st);
        w->steps++;
        const float c1 = 1.f - std::pow(b1, (float)w->steps), c2 = 1.f - std::pow(b2, (float)w->steps);
        adam_kernel<<<gsz(o.n), 256, 0, st>>>(w->th.p, w->m.p, w->v.p, w->grad.p, o.n, (float)lr, b1, b2, c1, c2);
        h->launches++;
        if (it == steps - 1 || (it % 50) == 0) {
            CCGF_CUDA_TRY(cudaMemcpyAsync(&last, w->loss.p, sizeof(double), cudaMemcpyDeviceToHost, st));
            CCGF_CUDA_TRY(cudaStreamSynchronize(st));
            if (!std::isfinite(last)) { set_last_error("warm-start training diverged"); return CCGF_ERR_NAN; }
        }
    }
    // validation on fresh rows: keep the learned correction only if it beats the baseline alone
    double vnet = 0, vbase = 0;
    const int nval = 8;
    h->launches += round_params(w->th.p, w->thr.p, w->F, w->H, w->bf16, st);
    for (int k = 0; k < nval; ++k) {
        CCGF_TRY(make_batch(k, 0x5bd1e995u));
        CCGF_CUDA_TRY(cudaMemsetAsync(w->loss.p, 0, sizeof(double), st));
        h->launches += backward(w->thr.p, w->F, w->H, rows, w->Fm.p, w->T.p, w->H1.p, w->H2.p, w->Y.p, w->dZ1.p, w->dZ2.p,
                                w->grad.p, w->loss.p, st);
        double l1 = 0;
        CCGF_CUDA_TRY(cudaMemcpyAsync(&l1, w->loss.p, sizeof(double), cudaMemcpyDeviceToHost, st));
        // the baseline's loss is the mean square of the targets (zero correction)
        std::vector<float> t(2 * rows);
        CCGF_CUDA_TRY(cudaMemcpyAsync(t.data(), w->T.p, sizeof(float) * 2 * rows, cudaMemcpyDeviceToHost, st));
        CCGF_CUDA_TRY(cudaStreamSynchronize(st));
        double l0 = 0;
        for (float x : t) l0 += (double)x * x;
        vnet += l1 / nval;
        vbase += l0 / rows / nval;
    }
    w->val_net = vnet;
    w->val_base = vbase;
    w->use_net = steps > 0 && vnet < vbase;
    if (!w->use_net) {
        CCGF_CUDA_TRY(cudaMemsetAsync(w->th.p + o.W3, 0, sizeof(float) * (2 * w->H + 2), st));   // baseline only
    }
    CCGF_CUDA_TRY(cudaGetLastError());
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(dall[0]);
    dfree(dall[1]);
    w->trained = true;
    if (final_loss) *final_loss = w->use_net ? vnet : vbase;
    return CCGF_OK;
}

void warmstart_losses(const ccgf_handle *h, double *val_net, double *val_base) {
    *val_net = h->ws ? h->ws->val_net : 0.0;
    *val_base = h->ws ? h->ws->val_base : 0.0;
}

// Standalone loss and gradient of the network (ABI helper for gradient checks).
extern "C" ccgf_status ccgf_mlp_loss_grad(int F, int H, long long rows, const float *theta, const float *X, const float *T,
                                          int bf16, double *loss, float *grad, void *stream) {
    if (F < 1 || H < 1 || rows < 1 || !theta || !X || !T || !loss || !grad) {
        set_last_error("invalid network sizes or NULL pointers");
        return CCGF_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    POff o = poff(F, H);
    DBuf<float> thr, H1, H2, Y, dZ1, dZ2;
    DBuf<double> dl;
    ccgf_status s = CCGF_OK;
    if ((s = dalloc(thr, o.n)) || (s = dalloc(H1, rows * H)) || (s = dalloc(H2, rows * H)) || (s = dalloc(Y, rows * 2)) ||
        (s = dalloc(dZ1, rows * H)) || (s = dalloc(dZ2, rows * H)) || (s = dalloc(dl, 1))) {
        dfree(thr); dfree(H1); dfree(H2); dfree(Y); dfree(dZ1); dfree(dZ2); dfree(dl);
        return s;
    }
    round_params(theta, thr.p, F, H, bf16, st);
    cudaMemsetAsync(dl.p, 0, sizeof(double), st);
    backward(thr.p, F, H, rows, X, T, H1.p, H2.p, Y.p, dZ1.p, dZ2.p, grad, dl.p, st);
    cudaMemcpyAsync(loss, dl.p, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    dfree(thr); dfree(H1); dfree(H2); dfree(Y); dfree(dZ1); dfree(dZ2); dfree(dl);
    if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); return CCGF_ERR_CUDA; }
    return CCGF_OK;
}

// Standalone forward pass (ABI helper): Y [rows][2].
extern "C" ccgf_status ccgf_mlp_forward(int F, int H, long long rows, const float *theta, const float *X, int bf16, float *Y,
                                        void *stream) {
    if (F < 1 || H < 1 || rows < 1 || !theta || !X || !Y) { set_last_error("invalid network sizes or NULL pointers"); return CCGF_ERR_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    POff o = poff(F, H);
    DBuf<float> thr, H1, H2;
    ccgf_status s = CCGF_OK;
    if ((s = dalloc(thr, o.n)) || (s = dalloc(H1, rows * H)) || (s = dalloc(H2, rows * H))) {
        dfree(thr); dfree(H1); dfree(H2);
        return s;
    }
    round_params(theta, thr.p, F, H, bf16, st);
    forward(thr.p, F, H, rows, X, H1.p, H2.p, Y, st);
    cudaError_t e = cudaStreamSynchronize(st);
    dfree(thr); dfree(H1); dfree(H2);
    if (e != cudaSuccess) { set_last_error(cudaGetErrorString(e)); return CCGF_ERR_CUDA; }
    return CCGF_OK;
}

// Copy out the trained parameters (host array of ccgf_mlp_param_count floats).
extern "C" long long ccgf_mlp_param_count(int F, int H) { return poff(F, H).n; }
