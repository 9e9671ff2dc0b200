// Build of the similarity-transformed Hamiltonian blocks (Eq. 5) used by the
// EOM-IP/EA-CCSD sigma vectors, in FP64, by direct per-element kernels.
//
// T1 is folded into the integrals: with X = 1 - t and Y = 1 + t (t[a,i] = t1[i,a])
// the dressed factors are L~[k1,k2,Q] = X(k1) L[k1,k2,Q] Y(k2), the dressed Fock
// matrix is X h Y + 2J~ - K~ with h = diag(e) - 2J + K, and every H_bar block is
// the T2-only expression in the dressed integrals. Each output element is written
// straight into the GEMM-ready layout the sigma plans read.
#include "ccgf_internal.h"
#include <cmath>
#include <algorithm>
#include <vector>

namespace {

struct Dims {
    int nk, o, v, n, Q;
    const int *kadd, *ksub;
};

__device__ __forceinline__ int kplus(const Dims &D, int a, int b) { return D.kadd[a * D.nk + b]; }
__device__ __forceinline__ int kminus(const Dims &D, int a, int b) { return D.ksub[a * D.nk + b]; }
__device__ __forceinline__ int kc3(const Dims &D, int k1, int k2, int k3) { return kplus(D, kminus(D, k1, k2), k3); }

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void cacc(double2 &acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// L[k1][k2][Q][p][q]
__device__ __forceinline__ i64 Lidx(const Dims &D, int k1, int k2, int q, int p, int r) {
    return ((((i64)k1 * D.nk + k2) * D.Q + q) * D.n + p) * D.n + r;
}
// chemist g[k1][k2][k3][p][q][r][s]
__device__ __forceinline__ i64 gidx(const Dims &D, int k1, int k2, int k3, int p, int q, int r, int s) {
    i64 n = D.n;
    return (((((((i64)k1 * D.nk + k2) * D.nk + k3) * n + p) * n + q) * n + r) * n + s);
}
// physicist <p kp, q kq | r kr, s ks> = (p r | q s) = g[kp][kr][kq][p][r][q][s]
__device__ __forceinline__ double2 PH(const Dims &D, const double2 *g, int kp, int kq, int kr, int p, int q, int r, int s) {
    return g[gidx(D, kp, kr, kq, p, r, q, s)];
}
// t2[ki][kj][ka][i][j][a][b]
__device__ __forceinline__ i64 tidx(const Dims &D, int ki, int kj, int ka, int i, int j, int a, int b) {
    return (((((((i64)ki * D.nk + kj) * D.nk + ka) * D.o + i) * D.o + j) * D.v + a) * D.v + b);
}

#define GRID_STRIDE(idx, total) for (i64 idx = (i64)blockIdx.x * blockDim.x + threadIdx.x; idx < (total); idx += (i64)gridDim.x * blockDim.x)

// ---------------------------------------------------------------- dressing
// L~[p,q] = M[p,q] - [p virt] sum_i t1[k1][i,p] M[i,q],  M = L Y(k2)
__global__ void dress_L_kernel(Dims D, const double2 *L, const double2 *t1, double2 *Ld) {
    const int n = D.n, o = D.o, v = D.v;
    i64 total = (i64)D.nk * D.nk * D.Q * n * n;
    GRID_STRIDE(idx, total) {
        int q = idx % n;
        int p = (idx / n) % n;
        int Qi = (idx / ((i64)n * n)) % D.Q;
        int k2 = (idx / ((i64)n * n * D.Q)) % D.nk;
        int k1 = idx / ((i64)n * n * D.Q * D.nk);
        auto M = [&](int pp) -> double2 {
            double2 m = L[Lidx(D, k1, k2, Qi, pp, q)];
            if (q < o)
                for (int a = 0; a < v; ++a) cacc(m, L[Lidx(D, k1, k2, Qi, pp, o + a)], t1[((i64)k2 * o + q) * v + a]);
            return m;
        };
        double2 r = M(p);
        if (p >= o) {
            for (int i = 0; i < o; ++i) {
                double2 mi = M(i);
                double2 tt = t1[((i64)k1 * o + i) * v + (p - o)];
                r = csub(r, cmul(tt, mi));
            }
        }
        Ld[idx] = r;
    }
}

// d[Q] = sum_{k,j} L[k,k,Q][j,j]
__global__ void diag_sum_kernel(Dims D, const double2 *L, double2 *d) {
    for (int q = threadIdx.x; q < D.Q; q += blockDim.x) {
        double2 acc = make_double2(0, 0);
        for (int k = 0; k < D.nk; ++k)
            for (int j = 0; j < D.o; ++j) acc = cadd(acc, L[Lidx(D, k, k, q, j, j)]);
        d[q] = acc;
    }
}

// J[k][p,q] = sum_Q L[k,k,Q][p,q] d[Q];  K[k][p,q] = sum_{kj,Q,j} L[k,kj,Q][p,j] L[kj,k,Q][j,q]
__device__ double2 jk_combo(const Dims &D, const double2 *L, const double2 *d, int k, int p, int q) {
    double2 J = make_double2(0, 0), K = make_double2(0, 0);
    for (int Qi = 0; Qi < D.Q; ++Qi) {
        cacc(J, L[Lidx(D, k, k, Qi, p, q)], d[Qi]);
        for (int kj = 0; kj < D.nk; ++kj)
            for (int j = 0; j < D.o; ++j) cacc(K, L[Lidx(D, k, kj, Qi, p, j)], L[Lidx(D, kj, k, Qi, j, q)]);
    }
    return csub(cscale(J, 2.0), K);   // 2J - K
}

__global__ void core_h_kernel(Dims D, const double *eps, const double2 *L, const double2 *d, double2 *h) {
    i64 total = (i64)D.nk * D.n * D.n;
    GRID_STRIDE(idx, total) {
        int q = idx % D.n, p = (idx / D.n) % D.n, k = idx / ((i64)D.n * D.n);
        double2 r = csub(make_double2(p == q ? eps[k * D.n + p] : 0.0, 0.0), jk_combo(D, L, d, k, p, q));
        h[idx] = r;
    }
}

// f~ = X h Y + 2J~ - K~
__global__ void dressed_fock_kernel(Dims D, const double2 *h, const double2 *t1, const double2 *Ld, const double2 *dd, double2 *f) {
    const int n = D.n, o = D.o, v = D.v;
    i64 total = (i64)D.nk * n * n;
    GRID_STRIDE(idx, total) {
        int q = idx % n, p = (idx / n) % n, k = idx / ((i64)n * n);
        const double2 *hk = h + (i64)k * n * n;
        auto HY = [&](int pp) -> double2 {
            double2 m = hk[pp * n + q];
            if (q < o)
                for (int a = 0; a < v; ++a) cacc(m, hk[pp * n + o + a], t1[((i64)k * o + q) * v + a]);
            return m;
        };
        double2 r = HY(p);
        if (p >= o)
            for (int i = 0; i < o; ++i) r = csub(r, cmul(t1[((i64)k * o + i) * v + (p - o)], HY(i)));
        r = cadd(r, jk_combo(D, Ld, dd, k, p, q));
        f[idx] = r;
    }
}

// g~[k1,k2,k3][p,q,r,s] = sum_Q L~[k1,k2,Q][p,q] L~[k3,k4,Q][r,s], k4 = k1 - k2 + k3
__global__ void eri_kernel(Dims D, const double2 *Ld, double2 *g) {
    const int n = D.n;
    i64 n4 = (i64)n * n * n * n;
    i64 total = (i64)D.nk * D.nk * D.nk * n4;
    GRID_STRIDE(idx, total) {
        i64 e = idx % n4;
        int s = e % n, r = (e / n) % n, q = (e / ((i64)n * n)) % n, p = e / ((i64)n * n * n);
        i64 kb = idx / n4;
        int k3 = kb % D.nk, k2 = (kb / D.nk) % D.nk, k1 = kb / ((i64)D.nk * D.nk);
        int k4 = kc3(D, k1, k2, k3);
        double2 acc = make_double2(0, 0);
        for (int Qi = 0; Qi < D.Q; ++Qi) cacc(acc, Ld[Lidx(D, k1, k2, Qi, p, q)], Ld[Lidx(D, k3, k4, Qi, r, s)]);
        g[idx] = acc;
    }
}

// ---------------------------------------------------------------- one-body blocks
__global__ void fock_blocks_kernel(Dims D, const double2 *g, const double2 *f, const double2 *t2,
                                   double2 *Foo, double2 *Fvv, double2 *Fov) {
    const int n = D.n, o = D.o, v = D.v, nk = D.nk;
    i64 per_k = (i64)o * o + (i64)v * v + (i64)o * v;
    i64 total = nk * per_k;
    GRID_STRIDE(idx, total) {
        int k = idx / per_k;
        i64 e = idx % per_k;
        const double2 *fk = f + (i64)k * n * n;
        if (e < (i64)o * o) {
            int m = e / o, i = e % o;
            double2 acc = fk[m * n + i];
            for (int kn = 0; kn < nk; ++kn)
                for (int ke = 0; ke < nk; ++ke) {
                    int kf = kc3(D, k, ke, kn);
                    for (int nn = 0; nn < o; ++nn)
                        for (int ee = 0; ee < v; ++ee)
                            for (int ff = 0; ff < v; ++ff) {
                                double2 w = csub(cscale(PH(D, g, k, kn, ke, m, nn, o + ee, o + ff), 2.0),
                                                 PH(D, g, k, kn, kf, m, nn, o + ff, o + ee));
                                cacc(acc, w, t2[tidx(D, k, kn, ke, i, nn, ee, ff)]);
                            }
                }
            Foo[(i64)k * o * o + m * o + i] = acc;
        } else if (e < (i64)o * o + (i64)v * v) {
            e -= (i64)o * o;
            int a = e / v, ee = e % v;
            double2 acc = fk[(o + a) * n + o + ee];
            for (int km = 0; km < nk; ++km)
                for (int kn = 0; kn < nk; ++kn) {
                    int kf = kc3(D, km, k, kn);
                    for (int m = 0; m < o; ++m)
                        for (int nn = 0; nn < o; ++nn)
                            for (int ff = 0; ff < v; ++ff) {
                                double2 w = csub(cscale(PH(D, g, km, kn, k, m, nn, o + ee, o + ff), 2.0),
                                                 PH(D, g, km, kn, kf, m, nn, o + ff, o + ee));
                                double2 t = t2[tidx(D, km, kn, k, m, nn, a, ff)];
                                acc = csub(acc, cmul(w, t));
                            }
                }
            Fvv[(i64)k * v * v + a * v + ee] = acc;
        } else {
            e -= (i64)o * o + (i64)v * v;
            int m = e / v, ee = e % v;
            Fov[(i64)k * o * v + m * v + ee] = fk[m * n + o + ee];
        }
    }
}

// ---------------------------------------------------------------- two-body blocks
// WvvvvP[ka][kb][a][b][ke][e][f] = <ab|ef> + sum_{km,m,n} <mn|ef> t[km,kn,ka][m,n,a,b]
__global__ void wvvvv_kernel(Dims D, const double2 *g, const double2 *t2, double2 *out) {
    const int o = D.o, v = D.v, nk = D.nk;
    i64 total = (i64)nk * nk * v * v * nk * v * v;
    GRID_STRIDE(idx, total) {
        i64 r = idx;
        int f = r % v; r /= v;
        int e = r % v; r /= v;
        int ke = r % nk; r /= nk;
        int b = r % v; r /= v;
        int a = r % v; r /= v;
        int kb = r % nk; r /= nk;
        int ka = (int)r;
        double2 acc = PH(D, g, ka, kb, ke, o + a, o + b, o + e, o + f);
        for (int km = 0; km < nk; ++km) {
            int kn = kc3(D, ka, km, kb);
            for (int m = 0; m < o; ++m)
                for (int nn = 0; nn < o; ++nn)
                    cacc(acc, PH(D, g, km, kn, ke, m, nn, o + e, o + f), t2[tidx(D, km, kn, ka, m, nn, a, b)]);
        }
        out[idx] = acc;
    }
}

// WvvvoP[ka][kb][ke][j][a][b][e] = Wvvvo[ka,kb,ke][a,b,e,j]
__global__ void wvvvo_kernel(Dims D, const double2 *g, const double2 *t2, const double2 *Fov, double2 *out) {
    const int o = D.o, v = D.v, nk = D.nk;
    i64 total = (i64)nk * nk * nk * o * v * v * v;
    GRID_STRIDE(idx, total) {
        i64 r = idx;
        int e = r % v; r /= v;
        int b = r % v; r /= v;
        int a = r % v; r /= v;
        int j = r % o; r /= o;
        int ke = r % nk; r /= nk;
        int kb = r % nk; r /= nk;
        int ka = (int)r;
        int kj = kc3(D, ka, ke, kb);
        const int A = o + a, B = o + b, E = o + e;
        double2 acc = PH(D, g, ka, kb, ke, A, B, E, j);
        for (int km = 0; km < nk; ++km) {
            int kn = kc3(D, ka, km, kb);
            for (int m = 0; m < o; ++m)
                for (int nn = 0; nn < o; ++nn) cacc(acc, PH(D, g, km, kn, ke, m, nn, E, j), t2[tidx(D, km, kn, ka, m, nn, a, b)]);
        }
        for (int m = 0; m < o; ++m) acc = csub(acc, cmul(Fov[((i64)ke * o + m) * v + e], t2[tidx(D, ke, kj, ka, m, j, a, b)]));
        for (int km = 0; km < nk; ++km) {
            int kf2 = kc3(D, km, ke, ka);   // km + ka - ke
            for (int m = 0; m < o; ++m)
                for (int f = 0; f < v; ++f) {
                    const int F = o + f;
                    // - <m b|e f> t[km,kj,ka][m,j,a,f]
                    acc = csub(acc, cmul(PH(D, g, km, kb, ke, m, B, E, F), t2[tidx(D, km, kj, ka, m, j, a, f)]));
                    double2 mafe = PH(D, g, km, ka, kf2, m, A, F, E);
                    double2 maef = PH(D, g, km, ka, ke, m, A, E, F);
                    // + (2<ma|fe> - <ma|ef>) t[km,kj,kf2][m,j,f,b] - <ma|fe> t[km,kj,kb][m,j,b,f]
                    cacc(acc, csub(cscale(mafe, 2.0), maef), t2[tidx(D, km, kj, kf2, m, j, f, b)]);
                    acc = csub(acc, cmul(mafe, t2[tidx(D, km, kj, kb, m, j, b, f)]));
                }
        }
        out[idx] = acc;
    }
}

// Wovvo / Wovov in the layout [kx][kj][km][j][x][m][e] (ke = km + kx - kj):
//   W1 = 2 Wovvo - Wovov, W2 = -Wovvo, WN = -Wovov
__global__ void wovvo_kernel(Dims D, const double2 *g, const double2 *t2, double2 *W1, double2 *W2, double2 *WN) {
    const int o = D.o, v = D.v, nk = D.nk;
    i64 total = (i64)nk * nk * nk * o * v * o * v;
    GRID_STRIDE(idx, total) {
        i64 r = idx;
        int e = r % v; r /= v;
        int m = r % o; r /= o;
        int x = r % v; r /= v;
        int j = r % o; r /= o;
        int km = r % nk; r /= nk;
        int kj = r % nk; r /= nk;
        int kx = (int)r;
        int ke = kc3(D, km, kj, kx);
        const int X = o + x, E = o + e;
        // Wovvo[km,kx,ke][m,x,e,j] = <mx|ej> + sum_{kn,n,f} [(2<mn|ef>-<mn|fe>) t[kj,kn,kx][j,n,x,f] - <mn|ef> t[kj,kn,kf][j,n,f,x]]
        double2 wvo = PH(D, g, km, kx, ke, m, X, E, j);
        // Wovov[km,kx,kj][m,x,j,e] = <mx|je> - sum_{kn,n,f} <mn|fe> t[kj,kn,kf][j,n,f,x]
        double2 wov = PH(D, g, km, kx, kj, m, X, j, E);
        for (int kn = 0; kn < nk; ++kn) {
            int kf = kc3(D, km, ke, kn);
            for (int nn = 0; nn < o; ++nn)
                for (int f = 0; f < v; ++f) {
                    const int F = o + f;
                    double2 mnef = PH(D, g, km, kn, ke, m, nn, E, F);
                    double2 mnfe = PH(D, g, km, kn, kf, m, nn, F, E);
                    cacc(wvo, csub(cscale(mnef, 2.0), mnfe), t2[tidx(D, kj, kn, kx, j, nn, x, f)]);
                    double2 tjnfx = t2[tidx(D, kj, kn, kf, j, nn, f, x)];
                    wvo = csub(wvo, cmul(mnef, tjnfx));
                    wov = csub(wov, cmul(mnfe, tjnfx));
                }
        }
        W1[idx] = csub(cscale(wvo, 2.0), wov);
        W2[idx] = make_double2(-wvo.x, -wvo.y);
        WN[idx] = make_double2(-wov.x, -wov.y);
    }
}

// UvovvP[K][a][km][ke][m][e][f] = 2<aK m|e f> - <a m|f e>,  kf = K + km - ke
__global__ void uvovv_kernel(Dims D, const double2 *g, double2 *out) {
    const int o = D.o, v = D.v, nk = D.nk;
    i64 total = (i64)nk * v * nk * nk * o * v * v;
    GRID_STRIDE(idx, total) {
        i64 r = idx;
        int f = r % v; r /= v;
        int e = r % v; r /= v;
        int m = r % o; r /= o;
        int ke = r % nk; r /= nk;
        int km = r % nk; r /= nk;
        int a = r % v; r /= v;
        int K = (int)r;
        int kf = kc3(D, K, ke, km);
        double2 w = csub(cscale(PH(D, g, K, km, ke, o + a, m, o + e, o + f), 2.0), PH(D, g, K, km, kf, o + a, m, o + f, o + e));
        out[idx] = w;
    }
}

// U_oovv for the three-body terms: EA  [K][m][kn][ke][n][e][f]  (m at K, kf = K + kn - ke)
//                                   IP  [K][e][km][kn][m][n][f]  (e at K, kf = km + kn - K)
// value 2<mn|ef> - <mn|fe>
__global__ void uoovv_kernel(Dims D, const double2 *g, double2 *out_ea, double2 *out_ip) {
    const int o = D.o, v = D.v, nk = D.nk;
    i64 total = (i64)nk * o * nk * nk * o * v * v;
    GRID_STRIDE(idx, total) {
        i64 r = idx;
        int f = r % v; r /= v;
        int e = r % v; r /= v;
        int nn = r % o; r /= o;
        int ke = r % nk; r /= nk;
        int kn = r % nk; r /= nk;
        int m = r % o; r /= o;
        int K = (int)r;
        int kf = kc3(D, K, ke, kn);
        out_ea[idx] = csub(cscale(PH(D, g, K, kn, ke, m, nn, o + e, o + f), 2.0), PH(D, g, K, kn, kf, m, nn, o + f, o + e));
    }
    i64 total2 = (i64)nk * v * nk * nk * o * o * v;
    GRID_STRIDE(idx, total2) {
        i64 r = idx;
        int f = r % v; r /= v;
        int nn = r % o; r /= o;
        int m = r % o; r /= o;
        int kn = r % nk; r /= nk;
        int km = r % nk; r /= nk;
        int e = r % v; r /= v;
        int K = (int)r;
        int kf = kc3(D, km, K, kn);
        out_ip[idx] = csub(cscale(PH(D, g, km, kn, K, m, nn, o + e, o + f), 2.0), PH(D, g, km, kn, kf, m, nn, o + f, o + e));
    }
}

// t2P_ea[K][kj][ka][j][a][b][m] = t2[K,kj,ka][m,j,a,b];  t2P_ip[ki][kj][K][i][j][a][e] = t2[ki,kj,K][i,j,e,a]
__global__ void t2perm_kernel(Dims D, const double2 *t2, double2 *tea, double2 *tip) {
    const int o = D.o, v = D.v, nk = D.nk;
    i64 total = (i64)nk * nk * nk * o * o * v * v;
    GRID_STRIDE(idx, total) {
        i64 r = idx;
        int m = r % o; r /= o;
        int b = r % v; r /= v;
        int a = r % v; r /= v;
        int j = r % o; r /= o;
        int k3 = r % nk; r /= nk;
        int k2 = r % nk; r /= nk;
        int k1 = (int)r;
        tea[idx] = t2[tidx(D, k1, k2, k3, m, j, a, b)];
    }
    GRID_STRIDE(idx, total) {
        i64 r = idx;
        int e = r % v; r /= v;
        int a = r % v; r /= v;
        int j = r % o; r /= o;
        int i = r % o; r /= o;
        int K = r % nk; r /= nk;
        int kj = r % nk; r /= nk;
        int ki = (int)r;
        tip[idx] = t2[tidx(D, ki, kj, K, i, j, e, a)];
    }
}

// WovooP[K][ki][kj][i][j][a][m] = Wovoo[K,ka,ki][m,a,i,j], ka = ki + kj - K
__global__ void wovoo_kernel(Dims D, const double2 *g, const double2 *t2, const double2 *Fov, double2 *out) {
    const int o = D.o, v = D.v, nk = D.nk;
    i64 total = (i64)nk * nk * nk * o * o * v * o;
    GRID_STRIDE(idx, total) {
        i64 r = idx;
        int m = r % o; r /= o;
        int b = r % v; r /= v;
        int j = r % o; r /= o;
        int i = r % o; r /= o;
        int kj = r % nk; r /= nk;
        int ki = r % nk; r /= nk;
        int K = (int)r;
        const int km = K;
        const int kb = kc3(D, ki, K, kj);
        const int B = o + b;
        double2 acc = PH(D, g, km, kb, ki, m, B, i, j);
        for (int ke = 0; ke < nk; ++ke)
            for (int e = 0; e < v; ++e)
                for (int f = 0; f < v; ++f)
                    cacc(acc, PH(D, g, km, kb, ke, m, B, o + e, o + f), t2[tidx(D, ki, kj, ke, i, j, e, f)]);
        for (int e = 0; e < v; ++e) cacc(acc, Fov[((i64)km * o + m) * v + e], t2[tidx(D, ki, kj, km, i, j, e, b)]);
        for (int kn = 0; kn < nk; ++kn) {
            int ke = kc3(D, km, ki, kn);
            int ke2 = kc3(D, km, kj, kn);
            for (int nn = 0; nn < o; ++nn)
                for (int e = 0; e < v; ++e) {
                    const int E = o + e;
                    double2 mnie = PH(D, g, km, kn, ki, m, nn, i, E);
                    double2 mnei = PH(D, g, km, kn, ke, m, nn, E, i);
                    cacc(acc, csub(cscale(mnie, 2.0), mnei), t2[tidx(D, kj, kn, kb, j, nn, b, e)]);
                    acc = csub(acc, cmul(mnie, t2[tidx(D, kj, kn, ke, j, nn, e, b)]));
                    acc = csub(acc, cmul(PH(D, g, km, kn, ke2, m, nn, E, j), t2[tidx(D, ki, kn, ke2, i, nn, e, b)]));
                }
        }
        out[idx] = acc;
    }
}

// WooooP[ki][kj][i][j][km][m][n] = Woooo[km,kn,ki][m,n,i,j], kn = ki + kj - km
__global__ void woooo_kernel(Dims D, const double2 *g, const double2 *t2, double2 *out) {
    const int o = D.o, v = D.v, nk = D.nk;
    i64 total = (i64)nk * nk * o * o * nk * o * o;
    GRID_STRIDE(idx, total) {
        i64 r = idx;
        int nn = r % o; r /= o;
        int m = r % o; r /= o;
        int km = r % nk; r /= nk;
        int j = r % o; r /= o;
        int i = r % o; r /= o;
        int kj = r % nk; r /= nk;
        int ki = (int)r;
        int kn = kc3(D, ki, km, kj);
        double2 acc = PH(D, g, km, kn, ki, m, nn, i, j);
        for (int ke = 0; ke < nk; ++ke)
            for (int e = 0; e < v; ++e)
                for (int f = 0; f < v; ++f)
                    cacc(acc, PH(D, g, km, kn, ke, m, nn, o + e, o + f), t2[tidx(D, ki, kj, ke, i, j, e, f)]);
        out[idx] = acc;
    }
}

// UooovP[K][i][km][kn][m][n][e] = 2<m n|i K, e> - <m n|e i K>,  ke = km + kn - K
__global__ void uooov_kernel(Dims D, const double2 *g, double2 *out) {
    const int o = D.o, v = D.v, nk = D.nk;
    i64 total = (i64)nk * o * nk * nk * o * o * v;
    GRID_STRIDE(idx, total) {
        i64 r = idx;
        int e = r % v; r /= v;
        int nn = r % o; r /= o;
        int m = r % o; r /= o;
        int kn = r % nk; r /= nk;
        int km = r % nk; r /= nk;
        int i = r % o; r /= o;
        int K = (int)r;
        int ke = kc3(D, km, K, kn);
        out[idx] = csub(cscale(PH(D, g, km, kn, K, m, nn, i, o + e), 2.0), PH(D, g, km, kn, ke, m, nn, o + e, i));
    }
}

// Pair-symmetric ladder blocks. For pair momentum s, representative pairs alpha = (ka, a, b)
// (kb = s - ka) are listed in reps[s][.] as (ka * v + a) * v + b: first the n_minus[s] pairs with
// ka*v+a < kb*v+b, then the fixed pairs (ka = kb, a = b). With Pi the pair swap,
//   Wp[s][alpha][beta] = W(alpha, beta) + W(alpha, Pi beta)   (beta non-fixed), W(alpha, beta) (beta fixed)
//   Wm[s][alpha][beta] = W(alpha, beta) - W(alpha, Pi beta)   (alpha, beta non-fixed)
// zero-padded to Pp x Pp and Pm x Pm.
__global__ void wpm_kernel(Dims D, const double2 *Wv, const int *reps, const int *npl, const int *nmi, int Pp, int Pm,
                           double2 *Wp, double2 *Wm) {
    const int v = D.v, nk = D.nk;
    const i64 v2 = (i64)v * v, row = (i64)nk * v2;
    const i64 totp = (i64)nk * Pp * Pp, totm = (i64)nk * Pm * Pm;
    GRID_STRIDE(idx, totp + totm) {
        const bool plus = idx < totp;
        const i64 e = plus ? idx : idx - totp;
        const int P = plus ? Pp : Pm;
        const int s = (int)(e / ((i64)P * P));
        const int al = (int)((e / P) % P), be = (int)(e % P);
        const int nlim = plus ? npl[s] : nmi[s];
        double2 out = make_double2(0, 0);
        if (al < nlim && be < nlim) {
            const int ra = reps[(i64)s * Pp + al], rb = reps[(i64)s * Pp + be];
            const int ka = ra / (int)v2, a = (ra / v) % v, bb = ra % v;
            const int kb = kminus(D, s, ka);
            const int ke = rb / (int)v2, ee = (rb / v) % v, ff = rb % v;
            const int kf = kminus(D, s, ke);
            const i64 arow = (((i64)ka * nk + kb) * v2 + (i64)a * v + bb) * row;
            const double2 w1 = Wv[arow + (i64)ke * v2 + (i64)ee * v + ff];
            const bool fixed_be = (ke == kf && ee == ff);
            if (fixed_be) out = w1;
            else {
                const double2 w2 = Wv[arow + (i64)kf * v2 + (i64)ff * v + ee];
                out = plus ? cadd(w1, w2) : csub(w1, w2);
            }
        }
        (plus ? Wp : Wm)[e] = out;
    }
}

__global__ void to_float_kernel(const double2 *a, float2 *b, i64 n) {
    GRID_STRIDE(idx, n) b[idx] = make_float2((float)a[idx].x, (float)a[idx].y);
}

__global__ void finite_check_kernel(const double *a, i64 n, int *flag) {
    GRID_STRIDE(idx, n) {
        if (!isfinite(a[idx])) atomicExch(flag, 1);
    }
}

inline unsigned grid_for(i64 total) {
    i64 g = ceil_div(total, 256);
    if (g > 152 * 64) g = 152 * 64;
    return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

ccgf_status build_intermediates(ccgf_handle *h, const ccgf_system *sys, cudaStream_t st) {
    const int nk = h->nk, o = h->o, v = h->v, n = h->n, Q = h->naux;
    CCGF_TRY(dalloc(h->kadd_d, nk * nk));
    CCGF_TRY(dalloc(h->ksub_d, nk * nk));
    CCGF_CUDA_TRY(cudaMemcpyAsync(h->kadd_d.p, h->km.add.data(), sizeof(int) * nk * nk, cudaMemcpyHostToDevice, st));
    CCGF_CUDA_TRY(cudaMemcpyAsync(h->ksub_d.p, h->km.sub.data(), sizeof(int) * nk * nk, cudaMemcpyHostToDevice, st));
    CCGF_TRY(dalloc(h->zero_tab, 3));
    CCGF_CUDA_TRY(cudaMemsetAsync(h->zero_tab.p, 0, 3 * sizeof(i64), st));
    Dims D{nk, o, v, n, Q, h->kadd_d.p, h->ksub_d.p};

    // finite-input check (host arrays were already copied to device by the caller)
    {
        DBuf<int> flag;
        CCGF_TRY(dalloc(flag, 1));
        CCGF_CUDA_TRY(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
        finite_check_kernel<<<grid_for(h->L.n * 2), 256, 0, st>>>((const double *)h->L.p, h->L.n * 2, flag.p);
        finite_check_kernel<<<grid_for(h->t2.n * 2), 256, 0, st>>>((const double *)h->t2.p, h->t2.n * 2, flag.p);
        finite_check_kernel<<<grid_for(h->t1.n * 2), 256, 0, st>>>((const double *)h->t1.p, h->t1.n * 2, flag.p);
        finite_check_kernel<<<grid_for(h->l2.n * 2), 256, 0, st>>>((const double *)h->l2.p, h->l2.n * 2, flag.p);
        finite_check_kernel<<<grid_for(h->l1.n * 2), 256, 0, st>>>((const double *)h->l1.p, h->l1.n * 2, flag.p);
        finite_check_kernel<<<grid_for(h->eps.n), 256, 0, st>>>(h->eps.p, h->eps.n, flag.p);
        int hflag = 0;
        CCGF_CUDA_TRY(cudaMemcpyAsync(&hflag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        CCGF_CUDA_TRY(cudaStreamSynchronize(st));
        dfree(flag);
        if (hflag) {
            set_last_error("non-finite value in the inputs");
            return CCGF_ERR_NAN;
        }
    }

    DBuf<double2> Ld, d, dd, hcore, f, g;
    CCGF_TRY(dalloc(Ld, h->L.n));
    CCGF_TRY(dalloc(d, Q));
    CCGF_TRY(dalloc(dd, Q));
    CCGF_TRY(dalloc(hcore, (i64)nk * n * n));
    CCGF_TRY(dalloc(f, (i64)nk * n * n));
    dress_L_kernel<<<grid_for(Ld.n), 256, 0, st>>>(D, h->L.p, h->t1.p, Ld.p);
    diag_sum_kernel<<<1, 256, 0, st>>>(D, h->L.p, d.p);
    diag_sum_kernel<<<1, 256, 0, st>>>(D, Ld.p, dd.p);
    core_h_kernel<<<grid_for(hcore.n), 256, 0, st>>>(D, h->eps.p, h->L.p, d.p, hcore.p);
    dressed_fock_kernel<<<grid_for(f.n), 256, 0, st>>>(D, hcore.p, h->t1.p, Ld.p, dd.p, f.p);
    i64 gn = (i64)nk * nk * nk * n * n * n * n;
    CCGF_TRY(dalloc(g, gn));
    eri_kernel<<<grid_for(gn), 256, 0, st>>>(D, Ld.p, g.p);

    auto &W = h->W;
    CCGF_TRY(dalloc(W[BUF_FOO], (i64)nk * o * o));
    CCGF_TRY(dalloc(W[BUF_FVV], (i64)nk * v * v));
    CCGF_TRY(dalloc(W[BUF_FOV], (i64)nk * o * v));
    fock_blocks_kernel<<<grid_for((i64)nk * (o * o + v * v + o * v)), 256, 0, st>>>(D, g.p, f.p, h->t2.p, W[BUF_FOO].p,
                                                                                     W[BUF_FVV].p, W[BUF_FOV].p);
    i64 nk3 = (i64)nk * nk * nk;
    CCGF_TRY(dalloc(W[BUF_WVVVV], nk3 * v * v * v * v));
    wvvvv_kernel<<<grid_for(W[BUF_WVVVV].n), 256, 0, st>>>(D, g.p, h->t2.p, W[BUF_WVVVV].p);
    {
        // representatives of the pair space of every pair momentum s (host), then W+ / W-
        const int v2 = v * v;
        std::vector<int> np(nk), nm(nk);
        std::vector<std::vector<int>> lists(nk);
        for (int s = 0; s < nk; ++s) {
            std::vector<int> nonfixed, fixed;
            for (int ka = 0; ka < nk; ++ka) {
                const int kb = h->km.s(s, ka);
                for (int a = 0; a < v; ++a)
                    for (int bb = 0; bb < v; ++bb) {
                        const int c1 = ka * v + a, c2 = kb * v + bb;
                        if (c1 < c2) nonfixed.push_back((ka * v + a) * v + bb);
                        else if (c1 == c2) fixed.push_back((ka * v + a) * v + bb);
                    }
            }
            nm[s] = (int)nonfixed.size();
            np[s] = (int)(nonfixed.size() + fixed.size());
            lists[s] = nonfixed;
            lists[s].insert(lists[s].end(), fixed.begin(), fixed.end());
        }
        int Pp = 0, Pm = 0;
        for (int s = 0; s < nk; ++s) {
            Pp = std::max(Pp, np[s]);
            Pm = std::max(Pm, nm[s]);
        }
        Pp = std::max(Pp, 1);
        Pm = std::max(Pm, 1);
        std::vector<int> reps((size_t)nk * Pp, 0);
        for (int s = 0; s < nk; ++s)
            for (int i = 0; i < np[s]; ++i) reps[(size_t)s * Pp + i] = lists[s][i];
        h->lad_np = np;
        h->lad_nm = nm;
        h->lad_Pp = Pp;
        h->lad_Pm = Pm;
        CCGF_TRY(dalloc(h->lad_reps, (i64)nk * Pp));
        CCGF_TRY(dalloc(h->lad_npl, nk));
        CCGF_TRY(dalloc(h->lad_nmi, nk));
        CCGF_CUDA_TRY(cudaMemcpyAsync(h->lad_reps.p, reps.data(), sizeof(int) * reps.size(), cudaMemcpyHostToDevice, st));
        CCGF_CUDA_TRY(cudaMemcpyAsync(h->lad_npl.p, np.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
        CCGF_CUDA_TRY(cudaMemcpyAsync(h->lad_nmi.p, nm.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
        CCGF_TRY(dalloc(W[BUF_WPLUS], (i64)nk * Pp * Pp));
        CCGF_TRY(dalloc(W[BUF_WMINUS], (i64)nk * Pm * Pm));
        wpm_kernel<<<grid_for((i64)nk * (Pp * (i64)Pp + Pm * (i64)Pm)), 256, 0, st>>>(
            D, W[BUF_WVVVV].p, h->lad_reps.p, h->lad_npl.p, h->lad_nmi.p, Pp, Pm, W[BUF_WPLUS].p, W[BUF_WMINUS].p);
        h->launches++;
        CCGF_CUDA_TRY(cudaGetLastError());
        CCGF_CUDA_TRY(cudaStreamSynchronize(st));
        dfree(W[BUF_WVVVV]);   // the ladder reads only W+ / W-
        (void)v2;
    }
    CCGF_TRY(dalloc(W[BUF_WVVVO], nk3 * o * v * v * v));
    wvvvo_kernel<<<grid_for(W[BUF_WVVVO].n), 256, 0, st>>>(D, g.p, h->t2.p, W[BUF_FOV].p, W[BUF_WVVVO].p);
    h->wov_seg = nk3 * o * o * v * v;
    CCGF_TRY(dalloc(W[BUF_WOV3], 3 * h->wov_seg));
    wovvo_kernel<<<grid_for(h->wov_seg), 256, 0, st>>>(D, g.p, h->t2.p, W[BUF_WOV3].p, W[BUF_WOV3].p + h->wov_seg,
                                                       W[BUF_WOV3].p + 2 * h->wov_seg);
    CCGF_TRY(dalloc(W[BUF_UVOVV], nk3 * o * v * v * v));
    uvovv_kernel<<<grid_for(W[BUF_UVOVV].n), 256, 0, st>>>(D, g.p, W[BUF_UVOVV].p);
    CCGF_TRY(dalloc(W[BUF_UOOVV_EA], nk3 * o * o * v * v));
    CCGF_TRY(dalloc(W[BUF_UOOVV_IP], nk3 * o * o * v * v));
    uoovv_kernel<<<grid_for(W[BUF_UOOVV_EA].n), 256, 0, st>>>(D, g.p, W[BUF_UOOVV_EA].p, W[BUF_UOOVV_IP].p);
    CCGF_TRY(dalloc(W[BUF_T2EA], nk3 * o * o * v * v));
    CCGF_TRY(dalloc(W[BUF_T2IP], nk3 * o * o * v * v));
    t2perm_kernel<<<grid_for(W[BUF_T2EA].n), 256, 0, st>>>(D, h->t2.p, W[BUF_T2EA].p, W[BUF_T2IP].p);
    CCGF_TRY(dalloc(W[BUF_WOVOO], nk3 * o * o * o * v));
    wovoo_kernel<<<grid_for(W[BUF_WOVOO].n), 256, 0, st>>>(D, g.p, h->t2.p, W[BUF_FOV].p, W[BUF_WOVOO].p);
    CCGF_TRY(dalloc(W[BUF_WOOOO], nk3 * o * o * o * o));
    woooo_kernel<<<grid_for(W[BUF_WOOOO].n), 256, 0, st>>>(D, g.p, h->t2.p, W[BUF_WOOOO].p);
    CCGF_TRY(dalloc(W[BUF_UOOOV], nk3 * o * o * o * v));
    uooov_kernel<<<grid_for(W[BUF_UOOOV].n), 256, 0, st>>>(D, g.p, W[BUF_UOOOV].p);
    CCGF_CUDA_TRY(cudaGetLastError());

    // FP32 copies of every GEMM operand
    for (int b = BUF_FOO; b < NBUF; ++b) {
        if (!W[b].p) continue;
        CCGF_TRY(dalloc(h->Wf[b], W[b].n));
        to_float_kernel<<<grid_for(W[b].n), 256, 0, st>>>(W[b].p, h->Wf[b].p, W[b].n);
        h->launches++;
    }
    CCGF_CUDA_TRY(cudaGetLastError());
    h->launches += 22;   // the fixed kernels of this function (finite checks, dressing, ERIs, blocks)
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(g);
    dfree(Ld);
    dfree(d);
    dfree(dd);
    dfree(hcore);
    dfree(f);
    return CCGF_OK;
}
