// Right-hand sides b = P a_bar |Phi0> and left vectors e = <Phi0|(1+Lambda) a_bar^(+) |mu>
// of the shifted systems (Eq. 6) and the contraction of Eq. 7, spin-adapted, at total
// momentum K. a_bar = e^-T a e^T: the T1 part mixes creators/annihilators with
// X = 1 - t, Y = 1 + t; the T2 part adds the 2h1p / 2p1h pieces.
//
//   IP rhs, orbital p:  occupied i:  r1 = unit(i)
//                       virtual a:   r1[k] = t1[K][k,a],  r2[kk,kl][k,l,d] = t2[kk,kl,K][k,l,a,d]
//   IP left, orbital q: occupied k:  e1[i] = d_ik - sum (2t[K,kl,kc][k,l,c,d] - t[K,kl,kd][k,l,d,c]) l2[K,kl,kc][i,l,c,d]
//                                            - sum_c t1[K][k,c] l1[K][i,c]
//                                    e2[ki,kj][i,j,a] = 2 d(ki=K,i=k) l1[kj][j,a] - d(kj=K,j=k) l1[ki][i,a]
//                                            - sum_c t1[K][k,c] (2 l2[ki,kj,K][i,j,c,a] - l2[ki,kj,ka][i,j,a,c])
//                       virtual c:   e1[i] = l1[K][i,c],  e2 = 2 l2[ki,kj,K][i,j,c,a] - l2[ki,kj,ka][i,j,a,c]
//   EA rhs, orbital q:  virtual c:   r1 = unit(c)
//                       occupied k:  r1[c] = -t1[K][k,c],  r2[kl,kc][l,c,d] = -t2[K,kl,kc][k,l,c,d]
//   EA left, orbital p: occupied i:  e1[a] = -l1[K][i,a],  e2[kj,ka][j,a,b] = l2[kj,K,ka][j,i,a,b] - 2 l2[K,kj,ka][i,j,a,b]
//                       virtual c:   e1[a] = d_ca - sum t2[kk,kl,K][k,l,c,d] (2 l2[kk,kl,K][k,l,a,d] - l2[kl,kk,K][l,k,a,d])
//                                            - sum_k t1[K][k,c] l1[K][k,a]
//                                    e2[kj,ka][j,a,b] = 2 d(ka=K,a=c) l1[kj][j,b] - d(kb=K,b=c) l1[kj][j,a]
//                                            + sum_k t1[K][k,c] (l2[kj,K,ka][j,k,a,b] - 2 l2[K,kj,ka][k,j,a,b])
#include "ccgf_internal.h"
#include <algorithm>

namespace {

struct VD {
    int nk, o, v;
    const int *kadd, *ksub;
    const double2 *t1, *t2, *l1, *l2;
};
__device__ __forceinline__ int kcv(const VD &D, int k1, int k2, int k3) {
    return D.kadd[D.ksub[k1 * D.nk + k2] * D.nk + k3];
}
__device__ __forceinline__ i64 t2i(const VD &D, int ki, int kj, int ka, int i, int j, int a, int b) {
    return (((((((i64)ki * D.nk + kj) * D.nk + ka) * D.o + i) * D.o + j) * D.v + a) * D.v + b);
}
__device__ __forceinline__ i64 t1i(const VD &D, int k, int i, int a) { return ((i64)k * D.o + i) * D.v + a; }
__device__ __forceinline__ double2 cm(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 ca(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cs(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

__global__ void rhs_kernel(VD D, int sector, int K, int p, double2 *out, i64 ld) {
    const int o = D.o, v = D.v, nk = D.nk;
    const i64 dim = sector == CCGF_SECTOR_IP ? o + (i64)nk * nk * o * o * v : v + (i64)nk * nk * o * v * v;
    for (i64 mu = (i64)blockIdx.x * blockDim.x + threadIdx.x; mu < dim; mu += (i64)gridDim.x * blockDim.x) {
        double2 r = make_double2(0, 0);
        if (sector == CCGF_SECTOR_IP) {
            if (mu < o) {
                if (p < o) r.x = (mu == p) ? 1.0 : 0.0;
                else r = D.t1[t1i(D, K, (int)mu, p - o)];
            } else if (p >= o) {
                i64 e = mu - o;
                int a = e % v; e /= v;
                int l = e % o; e /= o;
                int k = e % o; e /= o;
                int kl = e % nk;
                int kk = (int)(e / nk);
                r = D.t2[t2i(D, kk, kl, K, k, l, p - o, a)];
            }
        } else {
            if (mu < v) {
                if (p >= o) r.x = (mu == p - o) ? 1.0 : 0.0;
                else r = cs(D.t1[t1i(D, K, p, (int)mu)], -1.0);
            } else if (p < o) {
                i64 e = mu - v;
                int d = e % v; e /= v;
                int c = e % v; e /= v;
                int l = e % o; e /= o;
                int kc = e % nk;
                int kl = (int)(e / nk);
                r = cs(D.t2[t2i(D, K, kl, kc, p, l, c, d)], -1.0);
            }
        }
        out[mu * ld] = r;
    }
}

// Elementwise part of the left vectors (r2 block; r1 of the plain cases).
__global__ void left_kernel(VD D, int sector, int K, int q, double2 *out, i64 ld) {
    const int o = D.o, v = D.v, nk = D.nk;
    const i64 dim = sector == CCGF_SECTOR_IP ? o + (i64)nk * nk * o * o * v : v + (i64)nk * nk * o * v * v;
    for (i64 mu = (i64)blockIdx.x * blockDim.x + threadIdx.x; mu < dim; mu += (i64)gridDim.x * blockDim.x) {
        double2 r = make_double2(0, 0);
        if (sector == CCGF_SECTOR_IP) {
            if (mu < o) {
                int i = (int)mu;
                if (q < o) {
                    r.x = (i == q) ? 1.0 : 0.0;
                    for (int c = 0; c < v; ++c) r = ca(r, cs(cm(D.t1[t1i(D, K, q, c)], D.l1[t1i(D, K, i, c)]), -1.0));
                } else {
                    r = D.l1[t1i(D, K, i, q - o)];
                }
            } else {
                i64 e = mu - o;
                int a = e % v; e /= v;
                int j = e % o; e /= o;
                int i = e % o; e /= o;
                int kj = e % nk;
                int ki = (int)(e / nk);
                int ka = kcv(D, ki, K, kj);
                auto vir = [&](int c) -> double2 {
                    return ca(cs(D.l2[t2i(D, ki, kj, K, i, j, c, a)], 2.0), cs(D.l2[t2i(D, ki, kj, ka, i, j, a, c)], -1.0));
                };
                if (q < o) {
                    if (ki == K && i == q) r = ca(r, cs(D.l1[t1i(D, kj, j, a)], 2.0));
                    if (kj == K && j == q) r = ca(r, cs(D.l1[t1i(D, ki, i, a)], -1.0));
                    for (int c = 0; c < v; ++c) r = ca(r, cs(cm(D.t1[t1i(D, K, q, c)], vir(c)), -1.0));
                } else {
                    r = vir(q - o);
                }
            }
        } else {
            if (mu < v) {
                int a = (int)mu;
                if (q < o) {
                    r = cs(D.l1[t1i(D, K, q, a)], -1.0);
                } else {
                    int c = q - o;
                    r.x = (a == c) ? 1.0 : 0.0;
                    for (int k = 0; k < o; ++k) r = ca(r, cs(cm(D.t1[t1i(D, K, k, c)], D.l1[t1i(D, K, k, a)]), -1.0));
                }
            } else {
                i64 e = mu - v;
                int b = e % v; e /= v;
                int a = e % v; e /= v;
                int j = e % o; e /= o;
                int ka = e % nk;
                int kj = (int)(e / nk);
                int kb = kcv(D, K, ka, kj);
                auto occ = [&](int i) -> double2 {
                    return ca(D.l2[t2i(D, kj, K, ka, j, i, a, b)], cs(D.l2[t2i(D, K, kj, ka, i, j, a, b)], -2.0));
                };
                if (q < o) {
                    r = occ(q);
                } else {
                    int c = q - o;
                    if (ka == K && a == c) r = ca(r, cs(D.l1[t1i(D, kj, j, b)], 2.0));
                    if (kb == K && b == c) r = ca(r, cs(D.l1[t1i(D, kj, j, a)], -1.0));
                    for (int k = 0; k < o; ++k) r = ca(r, cm(D.t1[t1i(D, K, k, c)], occ(k)));
                }
            }
        }
        out[mu * ld] = r;
    }
}

// Reduction part of e1 (IP occupied q / EA virtual q): one block per output element.
//   IP: sum over (kl, kc, l, c, d): nk^2 nocc nvir^2 terms
//   EA: sum over (kk, kl, k, l, d): nk^2 nocc^2 nvir terms
__global__ void left_reduce_kernel(VD D, int sector, int K, int q, double2 *out, i64 ld) {
    const int o = D.o, v = D.v, nk = D.nk;
    const int elem = blockIdx.x;   // i (IP) or a (EA)
    const i64 total = sector == CCGF_SECTOR_IP ? (i64)nk * nk * o * v * v : (i64)nk * nk * o * o * v;
    double sx = 0, sy = 0;
    for (i64 t = threadIdx.x; t < total; t += blockDim.x) {
        double2 prod;
        if (sector == CCGF_SECTOR_IP) {
            // (2t[K,kl,kc][q,l,c,d] - t[K,kl,kd][q,l,d,c]) l2[K,kl,kc][i,l,c,d]
            i64 e = t;
            int d = e % v; e /= v;
            int c = e % v; e /= v;
            int l = e % o; e /= o;
            int kc = e % nk;
            int kl = (int)(e / nk);
            int kd = kcv(D, K, kc, kl);
            double2 tt = ca(cs(D.t2[t2i(D, K, kl, kc, q, l, c, d)], 2.0), cs(D.t2[t2i(D, K, kl, kd, q, l, d, c)], -1.0));
            prod = cm(tt, D.l2[t2i(D, K, kl, kc, elem, l, c, d)]);
        } else {
            // t2[kk,kl,K][k,l,c,d] (2 l2[kk,kl,K][k,l,a,d] - l2[kl,kk,K][l,k,a,d]), c = q - nocc
            i64 e = t;
            int d = e % v; e /= v;
            int l = e % o; e /= o;
            int k = e % o; e /= o;
            int kl = e % nk;
            int kk = (int)(e / nk);
            double2 ll = ca(cs(D.l2[t2i(D, kk, kl, K, k, l, elem, d)], 2.0), cs(D.l2[t2i(D, kl, kk, K, l, k, elem, d)], -1.0));
            prod = cm(D.t2[t2i(D, kk, kl, K, k, l, q - o, d)], ll);
        }
        sx += prod.x;
        sy += prod.y;
    }
    __shared__ double rx[256], ry[256];
    rx[threadIdx.x] = sx;
    ry[threadIdx.x] = sy;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            rx[threadIdx.x] += rx[threadIdx.x + s];
            ry[threadIdx.x] += ry[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double2 r = out[(i64)elem * ld];
        r.x -= rx[0];
        r.y -= ry[0];
        out[(i64)elem * ld] = r;
    }
}

}  // namespace

static VD make_vd(ccgf_handle *h) {
    return VD{h->nk, h->o, h->v, h->kadd_d.p, h->ksub_d.p, h->t1.p, h->W[BUF_T2].p, h->l1.p, h->l2.p};
}

ccgf_status make_rhs(ccgf_handle *h, int sector, int K, int p, double2 *out, i64 ld, cudaStream_t st) {
    VD D = make_vd(h);
    i64 dim = sector == CCGF_SECTOR_IP ? h->dim_ip : h->dim_ea;
    rhs_kernel<<<(unsigned)std::min<i64>(ceil_div(dim, 256), 4096), 256, 0, st>>>(D, sector, K, p, out, ld);
    h->launches++;
    CCGF_CUDA_TRY(cudaGetLastError());
    return CCGF_OK;
}

ccgf_status make_left(ccgf_handle *h, int sector, int K, int q, double2 *out, i64 ld, cudaStream_t st) {
    VD D = make_vd(h);
    i64 dim = sector == CCGF_SECTOR_IP ? h->dim_ip : h->dim_ea;
    left_kernel<<<(unsigned)std::min<i64>(ceil_div(dim, 256), 4096), 256, 0, st>>>(D, sector, K, q, out, ld);
    h->launches++;
    if (sector == CCGF_SECTOR_IP && q < h->o) {
        left_reduce_kernel<<<h->o, 256, 0, st>>>(D, sector, K, q, out, ld);
        h->launches++;
    }
    if (sector == CCGF_SECTOR_EA && q >= h->o) {
        left_reduce_kernel<<<h->v, 256, 0, st>>>(D, sector, K, q, out, ld);
        h->launches++;
    }
    CCGF_CUDA_TRY(cudaGetLastError());
    return CCGF_OK;
}
