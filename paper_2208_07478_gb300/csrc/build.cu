// Build of the similarity-transformed Hamiltonian blocks (Eq. 5) used by the EOM-IP/EA-CCSD
// sigma vectors, in FP64, from the density-fitting factors: no four-index integral tensor over
// all momenta is ever formed.
//
// T1 is folded into the integrals: with X = 1 - t and Y = 1 + t (t[a,i] = t1[i,a]) the dressed
// factors are L~[k1,k2,Q] = X(k1) L[k1,k2,Q] Y(k2), the dressed Fock matrix is X h Y + 2J~ - K~
// with h = diag(e) - 2J + K, and every H_bar block is the T2-only expression in the dressed
// integrals (p k1 q k2 | r k3 s k4) = sum_Q L~[k1,k2,Q][p,q] L~[k3,k4,Q][r,s] (k1 + k3 = k2 + k4).
//
// Integral classes that blocks need are formed by tensor GEMMs over Q (tgemm.cu):
//   (m e | n f)  [km][ke][kn][m][e][n][f]       nk^3 o^2 v^2   (kept in the direct form)
//   (m i | n e)  [km][ki][kn][m][i][n][e]       nk^3 o^3 v     (build only)
//   (m e | b f)  one km slice at a time         nk^2 o v^3     (build only)
// and the contractions with T2 of the ring, W_oooo and W_ovoo blocks are tensor GEMMs written
// straight into the GEMM-ready layouts the sigma plans read. The EA ladder is built per pair
// momentum s from (a e | b f) (plus, in the stored form, sum_mn <mn|ef> t_mn^ab) and folded at
// once into its pair-symmetric blocks W+ / W-, so no O(nk^3 v^4) array exists beyond one s.
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
// (m km e ke | n kn f kf) = OVOV[km][ke][kn][m][e][n][f], kf = km - ke + kn
__device__ __forceinline__ double2 ovov(const Dims &D, const double2 *g, int km, int ke, int kn, int m, int e, int nn, int f) {
    return g[((((((i64)km * D.nk + ke) * D.nk + kn) * D.o + m) * D.v + e) * D.o + nn) * D.v + f];
}
// (m km i ki | n kn e ke) = OOOV[km][ki][kn][m][i][n][e], ke = km - ki + kn
__device__ __forceinline__ double2 ooov(const Dims &D, const double2 *g, int km, int ki, int kn, int m, int i, int nn, int e) {
    return g[((((((i64)km * D.nk + ki) * D.nk + kn) * D.o + m) * D.o + i) * D.o + nn) * D.v + e];
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

// ---------------------------------------------------------------- one-body blocks
// Foo[k][m,i] = f[m,i] + sum (2<mn|ef> - <mn|fe>) t[k,kn,ke][i,n,e,f]
// Fvv[k][a,e] = f[a,e] - sum (2<mn|ef> - <mn|fe>) t[km,kn,k][m,n,a,f]
// Fov[k][m,e] = f[m,e];  with <m n|e f> = (m e|n f)
__global__ void fock_blocks_kernel(Dims D, const double2 *G, const double2 *f, const double2 *t2, double2 *Foo, double2 *Fvv,
                                   double2 *Fov) {
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
                                double2 w = csub(cscale(ovov(D, G, k, ke, kn, m, ee, nn, ff), 2.0), ovov(D, G, k, kf, kn, m, ff, nn, ee));
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
                                double2 w = csub(cscale(ovov(D, G, km, k, kn, m, ee, nn, ff), 2.0), ovov(D, G, km, kf, kn, m, ff, nn, ee));
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

// ---------------------------------------------------------------- two-body blocks (per element, small)
// U_oovv for the three-body terms: EA  [K][m][kn][ke][n][e][f]  (m at K, kf = K + kn - ke)
//                                   IP  [K][e][km][kn][m][n][f]  (e at K, kf = km + kn - K)
// value 2<mn|ef> - <mn|fe> = 2 (m e|n f) - (m f|n e)
__global__ void uoovv_kernel(Dims D, const double2 *G, double2 *out_ea, double2 *out_ip) {
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
        out_ea[idx] = csub(cscale(ovov(D, G, K, ke, kn, m, e, nn, f), 2.0), ovov(D, G, K, kf, kn, m, f, nn, e));
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
        out_ip[idx] = csub(cscale(ovov(D, G, km, K, kn, m, e, nn, f), 2.0), ovov(D, G, km, kf, kn, m, f, nn, e));
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

// Wovoo += sum_e Fov[K][m,e] t[ki,kj,K][i,j,e,b]   (layout [K][ki][kj][i][j][b][m])
__global__ void wovoo_fov_kernel(Dims D, const double2 *t2, const double2 *Fov, double2 *out) {
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
        double2 acc = out[idx];
        for (int e = 0; e < v; ++e) cacc(acc, Fov[((i64)K * o + m) * v + e], t2[tidx(D, ki, kj, K, i, j, e, b)]);
        out[idx] = acc;
    }
}

// UooovP[K][i][km][kn][m][n][e] = 2<m n|i K, e> - <m n|e i K> = 2 (m i|n e) - (n i|m e),  ke = km + kn - K
__global__ void uooov_kernel(Dims D, const double2 *G, double2 *out) {
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
        out[idx] = csub(cscale(ooov(D, G, km, K, kn, m, i, nn, e), 2.0), ooov(D, G, kn, K, km, nn, i, m, e));
    }
}

// U[km][ke][kn][m][e][n][f] = 2 (m e|n f) - (m f|n e)  (= 2<mn|ef> - <mn|fe>), kf = km - ke + kn
__global__ void ovov_combo_kernel(Dims D, const double2 *G, double2 *U) {
    const int o = D.o, v = D.v, nk = D.nk;
    i64 total = (i64)nk * nk * nk * o * v * o * v;
    GRID_STRIDE(idx, total) {
        i64 r = idx;
        int f = r % v; r /= v;
        int nn = r % o; r /= o;
        int e = r % v; r /= v;
        int m = r % o; r /= o;
        int kn = r % nk; r /= nk;
        int ke = r % nk; r /= nk;
        int km = (int)r;
        int kf = kc3(D, km, ke, kn);
        U[idx] = csub(cscale(G[idx], 2.0), ovov(D, G, km, kf, kn, m, f, nn, e));
    }
}

// ring blocks from P = Wovvo and Qv = Wovov (both in the layout [kx][kj][km][j][x][m][e]):
//   W1 = 2P - Qv, W2 = -P, WN = -Qv   (P, Qv are read from the W2 and WN slots)
__global__ void ring_combine_kernel(double2 *W1, double2 *W2, double2 *WN, i64 n) {
    GRID_STRIDE(idx, n) {
        const double2 p = W2[idx], q = WN[idx];
        W1[idx] = csub(cscale(p, 2.0), q);
        W2[idx] = make_double2(-p.x, -p.y);
        WN[idx] = make_double2(-q.x, -q.y);
    }
}

// Pair-symmetric ladder blocks of pair momentum s from Wt[ka][ke][a][b][e][f] = W(alpha, beta) with
// alpha = (ka, a, b), kb = s - ka, beta = (ke, e, f), kf = s - ke. Representatives reps[s][.] =
// (ka * v + a) * v + b: first the n_minus[s] pairs with ka*v+a < kb*v+b, then the fixed pairs.
//   Wp[s][alpha][beta] = W(alpha, beta) + W(alpha, Pi beta)   (beta non-fixed), W(alpha, beta) (beta fixed)
//   Wm[s][alpha][beta] = W(alpha, beta) - W(alpha, Pi beta)   (alpha, beta non-fixed)
// zero-padded to Pp x Pp and Pm x Pm.
__global__ void wpm_kernel(Dims D, int s, const double2 *Wt, const int *reps, const int *npl, const int *nmi, int Pp, int Pm,
                           double2 *Wp, double2 *Wm) {
    const int v = D.v, nk = D.nk;
    const i64 v2 = (i64)v * v;
    const i64 totp = (i64)Pp * Pp, totm = (i64)Pm * Pm;
    GRID_STRIDE(idx, totp + totm) {
        const bool plus = idx < totp;
        const i64 e = plus ? idx : idx - totp;
        const int P = plus ? Pp : Pm;
        const int al = (int)(e / P), be = (int)(e % P);
        const int nlim = plus ? npl[s] : nmi[s];
        double2 out = make_double2(0, 0);
        if (al < nlim && be < nlim) {
            const int ra = reps[(i64)s * Pp + al], rb = reps[(i64)s * Pp + be];
            const int ka = ra / (int)v2, a = (ra / v) % v, bb = ra % v;
            const int ke = rb / (int)v2, ee = (rb / v) % v, ff = rb % v;
            const int kf = kminus(D, s, ke);
            const double2 w1 = Wt[((((i64)ka * nk + ke) * v + a) * v + bb) * v2 + (i64)ee * v + ff];
            const bool fixed_be = (ke == kf && ee == ff);
            if (fixed_be) out = w1;
            else {
                const double2 w2 = Wt[((((i64)ka * nk + kf) * v + a) * v + bb) * v2 + (i64)ff * v + ee];
                out = plus ? cadd(w1, w2) : csub(w1, w2);
            }
        }
        (plus ? Wp + (i64)s * totp : Wm + (i64)s * totm)[e] = out;
    }
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

// largest element offset an index map reaches over [0, dim)
i64 imap_span(const IMap &m, i64 dim) {
    if (dim <= 0) return 0;
    const i64 inner = std::min<i64>(m.d2, dim);
    return ((dim - 1) / m.d2) * m.s1 + (inner - 1) * m.s2;
}

ccgf_status BuildGemm::run(const char *what, int M, int N, int K, int nred, IMap am, IMap ak, IMap bk, IMap bn, IMap cm, IMap cn,
                           const double2 *A, i64 lenA, const double2 *B, i64 lenB, double2 *C, i64 lenC,
                           const std::vector<i64> &oA, const std::vector<i64> &oB, const std::vector<i64> &oC, double alpha,
                           double beta) {
    const i64 batch = (i64)oC.size();
    if ((i64)oA.size() != batch * nred || (i64)oB.size() != batch * nred) {
        set_last_error(std::string("internal tensor GEMM with inconsistent tables: ") + what);
        return CCGF_ERR_INVALID_ARG;
    }
    if (batch == 0 || M <= 0 || N <= 0 || K <= 0) return CCGF_OK;
    const i64 sA = imap_span(am, M) + imap_span(ak, K), sB = imap_span(bk, K) + imap_span(bn, N),
              sC = imap_span(cm, M) + imap_span(cn, N);
    for (i64 i = 0; i < batch * nred; ++i)
        if (oA[i] < 0 || oA[i] + sA >= lenA || oB[i] < 0 || oB[i] + sB >= lenB) {
            set_last_error(std::string("internal tensor GEMM out of bounds (operands): ") + what);
            return CCGF_ERR_INVALID_ARG;
        }
    for (i64 b = 0; b < batch; ++b)
        if (oC[b] < 0 || oC[b] + sC >= lenC) {
            set_last_error(std::string("internal tensor GEMM out of bounds (output): ") + what);
            return CCGF_ERR_INVALID_ARG;
        }
    std::vector<i64> t;
    t.reserve(oA.size() + oB.size() + oC.size());
    t.insert(t.end(), oA.begin(), oA.end());
    t.insert(t.end(), oB.begin(), oB.end());
    t.insert(t.end(), oC.begin(), oC.end());
    DBuf<i64> d;
    CCGF_TRY(dalloc(d, (i64)t.size()));
    CCGF_CUDA_TRY(cudaMemcpyAsync(d.p, t.data(), sizeof(i64) * t.size(), cudaMemcpyHostToDevice, st));
    TGemm g{};
    g.M = M;
    g.N = N;
    g.K = K;
    g.nred = nred;
    g.batch = (int)batch;
    g.am = am;
    g.ak = ak;
    g.bk = bk;
    g.bn = bn;
    g.cm = cm;
    g.cn = cn;
    g.offA = d.p;
    g.offB = d.p + oA.size();
    g.offC = d.p + oA.size() + oB.size();
    g.alpha = make_double2(alpha, 0.0);
    g.beta = make_double2(beta, 0.0);
    h->launches += launch_tgemm<double>(g, A, B, C, st);
    keep.push_back(std::move(d));
    CCGF_CUDA_TRY(cudaGetLastError());
    return CCGF_OK;
}

ccgf_status build_intermediates(ccgf_handle *h, const ccgf_system *sys, const ccgf_options *opt, cudaStream_t st) {
    (void)sys;
    const int nk = h->nk, o = h->o, v = h->v, n = h->n, Q = h->naux;
    const i64 nk3 = (i64)nk * nk * nk, n2 = (i64)n * n, v2 = (i64)v * v, ov = (i64)o * v, o2 = (i64)o * o;
    CCGF_TRY(dalloc(h->kadd_d, nk * nk));
    CCGF_TRY(dalloc(h->ksub_d, nk * nk));
    CCGF_CUDA_TRY(cudaMemcpyAsync(h->kadd_d.p, h->km.add.data(), sizeof(int) * nk * nk, cudaMemcpyHostToDevice, st));
    CCGF_CUDA_TRY(cudaMemcpyAsync(h->ksub_d.p, h->km.sub.data(), sizeof(int) * nk * nk, cudaMemcpyHostToDevice, st));
    CCGF_TRY(dalloc(h->zero_tab, 3));
    CCGF_CUDA_TRY(cudaMemsetAsync(h->zero_tab.p, 0, 3 * sizeof(i64), st));
    Dims D{nk, o, v, n, Q, h->kadd_d.p, h->ksub_d.p};
    const auto &km = h->km;

    // stored or direct form of the O(nk^3 o v^3) terms: direct when storing them would take more
    // than 4 GB (or when asked)
    const int mode = opt ? opt->direct_terms : 0;
    const double big_bytes = 16.0 * (double)nk3 * o * v * v2;
    h->direct = mode == 2 || (mode == 0 && big_bytes > 4e9);

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
        h->launches += 6;
        int hflag = 0;
        CCGF_CUDA_TRY(cudaMemcpyAsync(&hflag, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        CCGF_CUDA_TRY(cudaStreamSynchronize(st));
        if (hflag) {
            set_last_error("non-finite value in the inputs");
            return CCGF_ERR_NAN;
        }
    }
    // T2 becomes a GEMM operand of the handle
    h->W[BUF_T2] = std::move(h->t2);
    const double2 *t2 = h->W[BUF_T2].p;
    const i64 lt2 = h->W[BUF_T2].n;
    auto &W = h->W;

    // dressed factors, Fock matrices
    DBuf<double2> d, dd, hcore, f;
    CCGF_TRY(dalloc(W[BUF_LD], h->L.n));
    const double2 *Ld = W[BUF_LD].p;
    const i64 lLd = W[BUF_LD].n;
    CCGF_TRY(dalloc(d, Q));
    CCGF_TRY(dalloc(dd, Q));
    CCGF_TRY(dalloc(hcore, (i64)nk * n2));
    CCGF_TRY(dalloc(f, (i64)nk * n2));
    dress_L_kernel<<<grid_for(lLd), 256, 0, st>>>(D, h->L.p, h->t1.p, W[BUF_LD].p);
    diag_sum_kernel<<<1, 256, 0, st>>>(D, h->L.p, d.p);
    diag_sum_kernel<<<1, 256, 0, st>>>(D, Ld, dd.p);
    core_h_kernel<<<grid_for(hcore.n), 256, 0, st>>>(D, h->eps.p, h->L.p, d.p, hcore.p);
    dressed_fock_kernel<<<grid_for(f.n), 256, 0, st>>>(D, hcore.p, h->t1.p, Ld, dd.p, f.p);
    h->launches += 5;
    CCGF_CUDA_TRY(cudaGetLastError());

    BuildGemm G{h, st, {}};
    auto LB = [&](int k1, int k2) -> i64 { return ((i64)k1 * nk + k2) * Q * n2; };
    auto TB = [&](int ki, int kj, int ka) -> i64 { return (((i64)ki * nk + kj) * nk + ka) * o2 * v2; };
    const IMap Qmap = imap_single(n2);

    // (m e | n f) [km][ke][kn][m][e][n][f], kf = km - ke + kn
    CCGF_TRY(dalloc(W[BUF_OVOV], nk3 * o2 * v2));
    double2 *OVOV = W[BUF_OVOV].p;
    const i64 lOVOV = W[BUF_OVOV].n;
    auto VB = [&](int a, int b, int c) -> i64 { return (((i64)a * nk + b) * nk + c) * o2 * v2; };
    {
        std::vector<i64> oA, oB, oC;
        for (int k1 = 0; k1 < nk; ++k1)
            for (int k2 = 0; k2 < nk; ++k2)
                for (int k3 = 0; k3 < nk; ++k3) {
                    oA.push_back(LB(k1, k2) + o);
                    oB.push_back(LB(k3, km.c(k1, k2, k3)) + o);
                    oC.push_back(VB(k1, k2, k3));
                }
        CCGF_TRY(G.run("(me|nf)", (int)ov, (int)ov, Q, 1, imap_pair(v, n, 1), Qmap, Qmap, imap_pair(v, n, 1), imap_single(ov),
                       imap_single(1), Ld, lLd, Ld, lLd, OVOV, lOVOV, oA, oB, oC, 1.0, 0.0));
    }
    // (m i | n e) [km][ki][kn][m][i][n][e], ke = km - ki + kn
    DBuf<double2> OOOVb;
    CCGF_TRY(dalloc(OOOVb, nk3 * o2 * ov));
    double2 *OOOV = OOOVb.p;
    const i64 lOOOV = OOOVb.n;
    auto OB = [&](int a, int b, int c) -> i64 { return (((i64)a * nk + b) * nk + c) * o2 * ov; };
    {
        std::vector<i64> oA, oB, oC;
        for (int k1 = 0; k1 < nk; ++k1)
            for (int k2 = 0; k2 < nk; ++k2)
                for (int k3 = 0; k3 < nk; ++k3) {
                    oA.push_back(LB(k1, k2));
                    oB.push_back(LB(k3, km.c(k1, k2, k3)) + o);
                    oC.push_back(OB(k1, k2, k3));
                }
        CCGF_TRY(G.run("(mi|ne)", (int)o2, (int)ov, Q, 1, imap_pair(o, n, 1), Qmap, Qmap, imap_pair(v, n, 1), imap_single(ov),
                       imap_single(1), Ld, lLd, Ld, lLd, OOOV, lOOOV, oA, oB, oC, 1.0, 0.0));
    }

    // one-body blocks
    CCGF_TRY(dalloc(W[BUF_FOO], (i64)nk * o2));
    CCGF_TRY(dalloc(W[BUF_FVV], (i64)nk * v2));
    CCGF_TRY(dalloc(W[BUF_FOV], (i64)nk * ov));
    fock_blocks_kernel<<<grid_for((i64)nk * (o2 + v2 + ov)), 256, 0, st>>>(D, OVOV, f.p, t2, W[BUF_FOO].p, W[BUF_FVV].p,
                                                                           W[BUF_FOV].p);
    h->launches++;

    // W_oooo:  WooooP[ki][kj][i][j][km][m][n] = Woooo[km,kn,ki][m,n,i,j] = (m i|n j) + sum <mn|ef> t_ij^ef
    {
        CCGF_TRY(dalloc(W[BUF_WOOOO], nk3 * o2 * o2));
        double2 *Wo = W[BUF_WOOOO].p;
        const i64 lWo = W[BUF_WOOOO].n;
        auto CB = [&](int ki, int kj, int kmm) -> i64 { return ((i64)ki * nk + kj) * o2 * nk * o2 + (i64)kmm * o2; };
        std::vector<i64> oA, oB, oC, tA, tB;
        for (int ki = 0; ki < nk; ++ki)
            for (int kj = 0; kj < nk; ++kj)
                for (int kmm = 0; kmm < nk; ++kmm) {
                    const int kn = km.c(ki, kmm, kj);
                    oA.push_back(LB(kmm, ki));
                    oB.push_back(LB(kn, kj));
                    oC.push_back(CB(ki, kj, kmm));
                    for (int ke = 0; ke < nk; ++ke) {
                        tA.push_back(VB(kmm, ke, kn));
                        tB.push_back(TB(ki, kj, ke));
                    }
                }
        // (m i | n j): rows (m, i), columns (n, j)
        CCGF_TRY(G.run("Woooo bare", (int)o2, (int)o2, Q, 1, imap_pair(o, n, 1), Qmap, Qmap, imap_pair(o, n, 1),
                       imap_pair(o, o, o * nk * o2), imap_pair(o, 1, nk * o2), Ld, lLd, Ld, lLd, Wo, lWo, oA, oB, oC, 1.0, 0.0));
        // sum_{ke,e,f} (m e|n f) t[ki,kj,ke][i,j,e,f]: rows (m, n), columns (i, j)
        CCGF_TRY(G.run("Woooo t2", (int)o2, (int)o2, (int)v2, nk, imap_pair(o, v * o * v, v), imap_pair(v, o * v, 1),
                       imap_pair(v, v, 1), imap_pair(o, o * v2, v2), imap_pair(o, o, 1), imap_pair(o, o * nk * o2, nk * o2), OVOV,
                       lOVOV, t2, lt2, Wo, lWo, tA, tB, oC, 1.0, 1.0));
    }

    // ring blocks [kx][kj][km][j][x][m][e], ke = km + kx - kj:  P = Wovvo into the W2 slot, Qv = Wovov
    // into the WN slot, then W1 = 2P - Qv, W2 = -P, WN = -Qv
    {
        h->wov_seg = nk3 * o2 * v2;
        const i64 seg = h->wov_seg;
        CCGF_TRY(dalloc(W[BUF_WOV3], 3 * seg));
        double2 *W1 = W[BUF_WOV3].p;
        const i64 lW = W[BUF_WOV3].n;
        auto RB = [&](int kx, int kj, int kmm) -> i64 { return (((i64)kx * nk + kj) * nk + kmm) * o2 * v2; };
        const IMap c_me = imap_pair(v, v, 1), c_jx = imap_pair(v, v * o * v, ov);
        std::vector<i64> aP, bP, aQ, bQ, oP, oQ;
        std::vector<i64> a1, b1, a2, b2;
        for (int kx = 0; kx < nk; ++kx)
            for (int kj = 0; kj < nk; ++kj)
                for (int kmm = 0; kmm < nk; ++kmm) {
                    const int ke = km.c(kmm, kj, kx);
                    aP.push_back(LB(kmm, ke) + o);               // (m e | x j)
                    bP.push_back(LB(kx, kj) + (i64)o * n);
                    oP.push_back(RB(kx, kj, kmm) + seg);
                    aQ.push_back(LB(kmm, kj));                   // (m j | x e)
                    bQ.push_back(LB(kx, ke) + (i64)o * n + o);
                    oQ.push_back(RB(kx, kj, kmm) + 2 * seg);
                    for (int kn = 0; kn < nk; ++kn) {
                        const int kf = km.c(kmm, ke, kn);
                        a1.push_back(VB(kmm, ke, kn));   // (m e | n f)
                        b1.push_back(TB(kj, kn, kx));    // t[kj,kn,kx][j,n,x,f]
                        a2.push_back(VB(kmm, kf, kn));   // (m f | n e)
                        b2.push_back(TB(kj, kn, kf));    // t[kj,kn,kf][j,n,f,x]
                    }
                }
        // bare integrals: P = (m e | x j) rows (m, e) columns (j, x); Qv = (m j | x e) rows (m, j) columns (x, e)
        CCGF_TRY(G.run("Wovvo bare", (int)ov, (int)ov, Q, 1, imap_pair(v, n, 1), Qmap, Qmap, imap_pair(v, 1, n), c_me, c_jx, Ld, lLd,
                       Ld, lLd, W1, lW, aP, bP, oP, 1.0, 0.0));
        CCGF_TRY(G.run("Wovov bare", (int)o2, (int)v2, Q, 1, imap_pair(o, n, 1), Qmap, Qmap, imap_pair(v, n, 1),
                       imap_pair(o, v, v * o * v), imap_pair(v, ov, 1), Ld, lLd, Ld, lLd, W1, lW, aQ, bQ, oQ, 1.0, 0.0));
        // rows (m, e), columns (j, x), K (n, f) over every kn:
        //   P += (2 (m e|n f) - (m f|n e)) t[kj,kn,kx][j,n,x,f] - (m e|n f) t[kj,kn,kf][j,n,f,x]
        //   Qv -= (m f|n e) t[kj,kn,kf][j,n,f,x]
        const IMap a_me = imap_pair(v, v * o * v, ov), a_nf = imap_pair(v, v, 1);
        const IMap a_me_x = imap_pair(v, v * o * v, 1), a_nf_x = imap_pair(v, v, ov);
        const IMap b_nf_1 = imap_pair(v, v2, 1), b_jx_1 = imap_pair(v, o * v2, v);
        const IMap b_nf_2 = imap_pair(v, v2, v), b_jx_2 = imap_pair(v, o * v2, 1);
        {
            // 2 (m e|n f) - (m f|n e) formed once (same layout as (m e|n f)), then one GEMM against t[kj,kn,kx]
            DBuf<double2> U;
            CCGF_TRY(dalloc(U, lOVOV));
            ovov_combo_kernel<<<grid_for(lOVOV), 256, 0, st>>>(D, OVOV, U.p);
            h->launches++;
            CCGF_TRY(G.run("Wovvo t2 (1)", (int)ov, (int)ov, (int)ov, nk, a_me, a_nf, b_nf_1, b_jx_1, c_me, c_jx, U.p, U.n, t2, lt2,
                           W1, lW, a1, b1, oP, 1.0, 1.0));
            CCGF_CUDA_TRY(cudaStreamSynchronize(st));
        }
        CCGF_TRY(G.run("Wovvo t2 (3)", (int)ov, (int)ov, (int)ov, nk, a_me, a_nf, b_nf_2, b_jx_2, c_me, c_jx, OVOV, lOVOV, t2, lt2, W1,
                       lW, a1, b2, oP, -1.0, 1.0));
        CCGF_TRY(G.run("Wovov t2", (int)ov, (int)ov, (int)ov, nk, a_me_x, a_nf_x, b_nf_2, b_jx_2, c_me, c_jx, OVOV, lOVOV, t2, lt2, W1,
                       lW, a2, b2, oQ, -1.0, 1.0));
        ring_combine_kernel<<<grid_for(seg), 256, 0, st>>>(W1, W1 + seg, W1 + 2 * seg, seg);
        h->launches++;
    }

    // W_ovoo:  WovooP[K][ki][kj][i][j][b][m] = Wovoo[K,kb,ki][m,b,i,j], kb = ki + kj - K
    {
        CCGF_TRY(dalloc(W[BUF_WOVOO], nk3 * o2 * ov));
        double2 *Wv = W[BUF_WOVOO].p;
        const i64 lWv = W[BUF_WOVOO].n;
        auto CB = [&](int K, int ki, int kj) -> i64 { return (((i64)K * nk + ki) * nk + kj) * o2 * ov; };
        const IMap c_mi = imap_pair(o, 1, o * v * o), c_bj = imap_pair(o, o, v * o);
        const IMap c_mb = imap_pair(v, 1, o), c_ij = imap_pair(o, o * v * o, v * o);
        const IMap c_jb = imap_pair(v, v * o, o), c_mj = imap_pair(o, 1, v * o), c_ib = imap_pair(v, o * v * o, o);
        std::vector<i64> aB, bB, cB;
        std::vector<i64> a1, a1x, b1, b2, a3, b3;
        for (int K = 0; K < nk; ++K)
            for (int ki = 0; ki < nk; ++ki)
                for (int kj = 0; kj < nk; ++kj) {
                    const int kb = km.c(ki, K, kj);
                    aB.push_back(LB(K, ki));                     // (m i | b j)
                    bB.push_back(LB(kb, kj) + (i64)o * n);
                    cB.push_back(CB(K, ki, kj));
                    for (int kn = 0; kn < nk; ++kn) {
                        const int ke = km.c(K, ki, kn);          // (m i | n e), e at ke
                        const int ke2 = km.c(K, kj, kn);         // (m e | n j), e at ke2
                        a1.push_back(OB(K, ki, kn));
                        a1x.push_back(OB(kn, ki, K));            // (n i | m e)
                        b1.push_back(TB(kj, kn, kb));            // t[kj,kn,kb][j,n,b,e]
                        b2.push_back(TB(kj, kn, ke));            // t[kj,kn,ke][j,n,e,b]
                        a3.push_back(OB(kn, kj, K));             // (n j | m e)
                        b3.push_back(TB(ki, kn, ke2));           // t[ki,kn,ke2][i,n,e,b]
                    }
                }
        CCGF_TRY(G.run("Wovoo bare", (int)o2, (int)ov, Q, 1, imap_pair(o, n, 1), Qmap, Qmap, imap_pair(o, n, 1), c_mi, c_bj, Ld, lLd,
                       Ld, lLd, Wv, lWv, aB, bB, cB, 1.0, 0.0));
        // + sum (2 (m i|n e) - (n i|m e)) t[kj,kn,kb][j,n,b,e]: rows (m, i), columns (j, b), K (n, e)
        const IMap a_mi = imap_pair(o, o * o * v, ov), a_ne = imap_pair(v, v, 1);
        const IMap a_mi_x = imap_pair(o, v, ov), a_ne_x = imap_pair(v, o * o * v, 1);
        CCGF_TRY(G.run("Wovoo ooov (1)", (int)o2, (int)ov, (int)ov, nk, a_mi, a_ne, imap_pair(v, v2, 1), imap_pair(v, o * v2, v), c_mi,
                       c_jb, OOOV, lOOOV, t2, lt2, Wv, lWv, a1, b1, cB, 2.0, 1.0));
        CCGF_TRY(G.run("Wovoo ooov (2)", (int)o2, (int)ov, (int)ov, nk, a_mi_x, a_ne_x, imap_pair(v, v2, 1), imap_pair(v, o * v2, v),
                       c_mi, c_jb, OOOV, lOOOV, t2, lt2, Wv, lWv, a1x, b1, cB, -1.0, 1.0));
        // - (m i|n e) t[kj,kn,ke][j,n,e,b]
        CCGF_TRY(G.run("Wovoo ooov (3)", (int)o2, (int)ov, (int)ov, nk, a_mi, a_ne, imap_pair(v, v2, v), imap_pair(v, o * v2, 1), c_mi,
                       c_jb, OOOV, lOOOV, t2, lt2, Wv, lWv, a1, b2, cB, -1.0, 1.0));
        // - (n j|m e) t[ki,kn,ke2][i,n,e,b]: rows (m, j), columns (i, b)
        CCGF_TRY(G.run("Wovoo ooov (4)", (int)o2, (int)ov, (int)ov, nk, imap_pair(o, v, ov), imap_pair(v, o * o * v, 1),
                       imap_pair(v, v2, v), imap_pair(v, o * v2, 1), c_mj, c_ib, OOOV, lOOOV, t2, lt2, Wv, lWv, a3, b3, cB, -1.0,
                       1.0));
        // + sum_e Fov[K][m,e] t[ki,kj,K][i,j,e,b]
        wovoo_fov_kernel<<<grid_for(lWv), 256, 0, st>>>(D, t2, W[BUF_FOV].p, Wv);
        h->launches++;
        // + sum_{ke,e,f} (m e|b f) t[ki,kj,ke][i,j,e,f], one K (= km) slice of (m e|b f) at a time
        DBuf<double2> S;
        CCGF_TRY(dalloc(S, (i64)nk * nk * ov * v2));
        for (int K = 0; K < nk; ++K) {
            std::vector<i64> sA, sB, sC, gA, gB, gC;
            for (int ke = 0; ke < nk; ++ke)
                for (int kb = 0; kb < nk; ++kb) {
                    const int kf = km.c(K, ke, kb);
                    sA.push_back(LB(K, ke) + o);
                    sB.push_back(LB(kb, kf) + (i64)o * n + o);
                    sC.push_back(((i64)ke * nk + kb) * ov * v2);
                }
            // S[ke][kb][m][e][b][f] = (m e|b f): rows (m, e), columns (b, f)
            CCGF_TRY(G.run("(me|bf) slice", (int)ov, (int)v2, Q, 1, imap_pair(v, n, 1), Qmap, Qmap, imap_pair(v, n, 1),
                           imap_pair(v, v * v2, v2), imap_pair(v, v, 1), Ld, lLd, Ld, lLd, S.p, S.n, sA, sB, sC, 1.0, 0.0));
            for (int ki = 0; ki < nk; ++ki)
                for (int kj = 0; kj < nk; ++kj) {
                    const int kb = km.c(ki, K, kj);
                    for (int ke = 0; ke < nk; ++ke) {
                        gA.push_back(((i64)ke * nk + kb) * ov * v2);
                        gB.push_back(TB(ki, kj, ke));
                    }
                    gC.push_back(CB(K, ki, kj));
                }
            // rows (m, b), columns (i, j), K (e, f)
            CCGF_TRY(G.run("Wovoo ovvv", (int)ov, (int)o2, (int)v2, nk, imap_pair(v, v * v2, v), imap_pair(v, v2, 1), imap_pair(v, v, 1),
                           imap_pair(o, o * v2, v2), c_mb, c_ij, S.p, S.n, t2, lt2, Wv, lWv, gA, gB, gC, 1.0, 1.0));
        }
        CCGF_CUDA_TRY(cudaStreamSynchronize(st));
        G.keep.clear();
    }

    // U blocks and permuted T2 (per element)
    CCGF_TRY(dalloc(W[BUF_UOOVV_EA], nk3 * o2 * v2));
    CCGF_TRY(dalloc(W[BUF_UOOVV_IP], nk3 * o2 * v2));
    uoovv_kernel<<<grid_for(W[BUF_UOOVV_EA].n), 256, 0, st>>>(D, OVOV, W[BUF_UOOVV_EA].p, W[BUF_UOOVV_IP].p);
    CCGF_TRY(dalloc(W[BUF_UOOOV], nk3 * o2 * ov));
    uooov_kernel<<<grid_for(W[BUF_UOOOV].n), 256, 0, st>>>(D, OOOV, W[BUF_UOOOV].p);
    CCGF_TRY(dalloc(W[BUF_T2EA], nk3 * o2 * v2));
    CCGF_TRY(dalloc(W[BUF_T2IP], nk3 * o2 * v2));
    t2perm_kernel<<<grid_for(W[BUF_T2EA].n), 256, 0, st>>>(D, t2, W[BUF_T2EA].p, W[BUF_T2IP].p);
    h->launches += 3;
    CCGF_CUDA_TRY(cudaGetLastError());
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    dfree(OOOVb);

    // stored form: UvovvP[K][a][km][ke][m][e][f] = 2<a K, m|e f> - <a m|f e> = 2 (a e|m f) - (a f|m e), kf = K + km - ke
    if (!h->direct) {
        CCGF_TRY(dalloc(W[BUF_UVOVV], nk3 * ov * v2));
        double2 *U = W[BUF_UVOVV].p;
        const i64 lU = W[BUF_UVOVV].n, nko = (i64)nk * nk * o * v2;
        std::vector<i64> cA, cB, xA, xB, oC;
        for (int K = 0; K < nk; ++K)
            for (int kmm = 0; kmm < nk; ++kmm)
                for (int ke = 0; ke < nk; ++ke) {
                    const int kf = km.c(K, ke, kmm);
                    cA.push_back(LB(K, ke) + (i64)o * n + o);      // (a e | m f)
                    cB.push_back(LB(kmm, kf) + o);
                    xA.push_back(LB(K, kf) + (i64)o * n + o);      // (a f | m e)
                    xB.push_back(LB(kmm, ke) + o);
                    oC.push_back((i64)K * v * nko + ((i64)kmm * nk + ke) * o * v2);
                }
        // Coulomb: rows (a, e), columns (m, f); exchange: rows (a, f), columns (m, e)
        CCGF_TRY(G.run("Uvovv (1)", (int)v2, (int)ov, Q, 1, imap_pair(v, n, 1), Qmap, Qmap, imap_pair(v, n, 1), imap_pair(v, nko, v),
                       imap_pair(v, v2, 1), Ld, lLd, Ld, lLd, U, lU, cA, cB, oC, 2.0, 0.0));
        CCGF_TRY(G.run("Uvovv (2)", (int)v2, (int)ov, Q, 1, imap_pair(v, n, 1), Qmap, Qmap, imap_pair(v, n, 1), imap_pair(v, nko, 1),
                       imap_pair(v, v2, v), Ld, lLd, Ld, lLd, U, lU, xA, xB, oC, -1.0, 1.0));
    }

    // EA ladder: per pair momentum s, Wt[ka][ke][a][b][e][f] = (a e|b f) (+ sum_{km,m,n} (m e|n f)
    // t[km,kn,ka][m,n,a,b] in the stored form), then the pair-symmetric blocks W+ / W- of s
    {
        std::vector<int> np(nk), nm(nk);
        std::vector<std::vector<int>> lists(nk);
        for (int s = 0; s < nk; ++s) {
            std::vector<int> nonfixed, fixed;
            for (int ka = 0; ka < nk; ++ka) {
                const int kb = km.s(s, ka);
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
        int Pp = 1, Pm = 1;
        for (int s = 0; s < nk; ++s) {
            Pp = std::max(Pp, np[s]);
            Pm = std::max(Pm, nm[s]);
        }
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
        DBuf<double2> Wt;
        CCGF_TRY(dalloc(Wt, (i64)nk * nk * v2 * v2));
        const i64 v3 = v2 * v;
        for (int s = 0; s < nk; ++s) {
            std::vector<i64> oA, oB, oC, tA, tB;
            for (int ka = 0; ka < nk; ++ka)
                for (int ke = 0; ke < nk; ++ke) {
                    const int kb = km.s(s, ka), kf = km.s(s, ke);
                    oA.push_back(LB(ka, ke) + (i64)o * n + o);
                    oB.push_back(LB(kb, kf) + (i64)o * n + o);
                    oC.push_back(((i64)ka * nk + ke) * v2 * v2);
                    for (int kmm = 0; kmm < nk; ++kmm) {
                        const int kn = km.c(ka, kmm, kb);
                        tA.push_back(TB(kmm, kn, ka));    // t[km,kn,ka][m,n,a,b]
                        tB.push_back(VB(kmm, ke, kn));    // (m e|n f)
                    }
                }
            // (a e | b f): rows (a, e), columns (b, f)
            CCGF_TRY(G.run("ladder (ae|bf)", (int)v2, (int)v2, Q, 1, imap_pair(v, n, 1), Qmap, Qmap, imap_pair(v, n, 1),
                           imap_pair(v, v3, v), imap_pair(v, v2, 1), Ld, lLd, Ld, lLd, Wt.p, Wt.n, oA, oB, oC, 1.0, 0.0));
            if (!h->direct) {
                // + sum_{km} sum_{m,n} t[km,kn,ka][m,n,a,b] (m e|n f): rows (a, b), columns (e, f), K (m, n)
                CCGF_TRY(G.run("ladder t2", (int)v2, (int)v2, (int)o2, nk, imap_single(1), imap_pair(o, o * v2, v2),
                               imap_pair(o, v * o * v, v), imap_pair(v, o * v, 1), imap_single(v2), imap_single(1), t2, lt2, OVOV,
                               lOVOV, Wt.p, Wt.n, tA, tB, oC, 1.0, 1.0));
            }
            wpm_kernel<<<grid_for((i64)Pp * Pp + (i64)Pm * Pm), 256, 0, st>>>(D, s, Wt.p, h->lad_reps.p, h->lad_npl.p, h->lad_nmi.p,
                                                                             Pp, Pm, W[BUF_WPLUS].p, W[BUF_WMINUS].p);
            h->launches++;
        }
        CCGF_CUDA_TRY(cudaGetLastError());
        CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    }
    G.keep.clear();
    if (!h->direct) dfree(W[BUF_OVOV]);   // the direct form's ladder T2 term reads it in every EA sigma

    // stored form: W_vvvo, formed by applying the EA r1 -> r2 terms to unit vectors
    if (!h->direct) CCGF_TRY(build_wvvvo_by_plan(h, st));
    CCGF_CUDA_TRY(cudaGetLastError());
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    return CCGF_OK;
}
