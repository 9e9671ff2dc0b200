// EOM-IP / EA-CCSD sigma vectors (Eq. 8 spaces, H_bar of Eq. 5) as plans of
// batched complex GEMMs and permutes over momentum-conserving k-blocks.
//
// Vectors inside the library are element-major: row mu of the EOM space, nv
// right-hand sides contiguous per row ([D][nv]). Every term of the spin-adapted
// sigma then is a batched GEMM whose N dimension is (orbital index x nv):
//
//   EA (total momentum K), r2[kj,ka][j,a,b], kb = K + kj - ka
//     s1[a]  = Fvv r1 + sum_{m,e} f_me (2 r2[km,K][m,a,e] - r2[km,km][m,e,a])
//              + sum (2<am|ef> - <am|fe>) r2[km,ke][m,e,f]
//     s2     = Wvvvo r1 + Fvv(a) r2 + Fvv(b) r2 - Foo(j) r2
//              + sum_km [(2 Wovvo - Wovov) R' - Wovvo Q'] - sum_km Wovov r2   (ring terms)
//              + sum_ke Wvvvv r2[kj,ke] - t2 . (sum (2<mn|ef> - <mn|fe>) r2)   (ladder, 3-body)
//   IP (total momentum K), r2[ki,kj][i,j,a], ka = ki + kj - K: the mirror terms
//     (Foo, Fov, 2<mn|ie> - <mn|ei>, Wovoo, Fvv, Foo(i), Foo(j), Woooo, ring, 3-body).
//
// Plans hold device offset tables (per batch entry and per momentum reduction),
// built once per (sector, K, nv) and replayed on every call; the same plan runs
// on the FP64 intermediates or on their FP32 copies.
#include "ccgf_internal.h"
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>

namespace {

struct PlanBuilder {
    SigmaPlan *P;
    std::vector<i64> off;   // host copy of the offset table
    const char *cur = "";   // label of the term being emitted

    i64 push(const std::vector<i64> &v) {
        i64 pos = (i64)off.size();
        off.insert(off.end(), v.begin(), v.end());
        return pos;
    }
    void gemm(int M, int N, int K, int nred, int a_buf, i64 rsA, i64 csA, const std::vector<i64> &oA, i64 rsB, i64 csB,
              const std::vector<i64> &oB, int c_buf, i64 rsC, i64 csC, const std::vector<i64> &oC, double alpha, double beta) {
        SigmaStep s{};
        s.name = cur;
        s.kind = STEP_GEMM;
        s.g.M = M;
        s.g.N = N;
        s.g.K = K;
        s.g.nred = nred;
        s.g.batch = (int)oC.size();
        s.g.rsA = rsA;
        s.g.csA = csA;
        s.g.rsB = rsB;
        s.g.csB = csB;
        s.g.rsC = rsC;
        s.g.csC = csC;
        s.g.alpha = make_double2(alpha, 0.0);
        s.g.beta = make_double2(beta, 0.0);
        s.a_buf = a_buf;
        s.c_buf = c_buf;
        s.offA_pos = push(oA);
        s.offB_pos = push(oB);
        s.offC_pos = push(oC);
        // row coordinates of the A blocks for the TMA-fed tensor-core path
        s.rowA_pos = -1;
        if (csA == 1 && rsA > 0) {
            std::vector<i64> rows;
            for (i64 a : oA) {
                if (a % rsA) break;
                rows.push_back(a / rsA);
            }
            if (rows.size() == oA.size()) s.rowA_pos = push(rows);
        }
        // distinct B blocks (slots) for the bulk-fed tensor-core path
        {
            std::map<i64, i64> slot_of;
            std::vector<i64> slots, src;
            for (i64 b : oB) {
                auto it = slot_of.find(b);
                if (it == slot_of.end()) {
                    it = slot_of.emplace(b, (i64)src.size()).first;
                    src.push_back(b);
                }
                slots.push_back(it->second);
            }
            s.nslots = (int)src.size();
            s.bslot_pos = push(slots);
            s.bsrc_pos = push(src);
        }
        P->steps.push_back(s);
    }
    // tensor GEMM (pair index maps); a_buf / b_buf: intermediate or BUF_SCRATCH, c_buf: BUF_Y or BUF_SCRATCH
    void tgemm(int M, int N, int K, int nred, int a_buf, IMap am, IMap ak, const std::vector<i64> &oA, int b_buf, IMap bk,
               IMap bn, const std::vector<i64> &oB, int c_buf, IMap cm, IMap cn, const std::vector<i64> &oC, double alpha,
               double beta) {
        SigmaStep s{};
        s.name = cur;
        s.kind = STEP_TGEMM;
        s.tg.M = M;
        s.tg.N = N;
        s.tg.K = K;
        s.tg.nred = nred;
        s.tg.batch = (int)oC.size();
        s.tg.am = am;
        s.tg.ak = ak;
        s.tg.bk = bk;
        s.tg.bn = bn;
        s.tg.cm = cm;
        s.tg.cn = cn;
        s.tg.alpha = make_double2(alpha, 0.0);
        s.tg.beta = make_double2(beta, 0.0);
        s.a_buf = a_buf;
        s.b_buf = b_buf;
        s.c_buf = c_buf;
        s.offA_pos = push(oA);
        s.offB_pos = push(oB);
        s.offC_pos = push(oC);
        s.rowA_pos = -1;
        P->steps.push_back(s);
    }
    // dims (outer..inner), source strides (scratch), destination strides
    void perm(std::vector<i64> dims, std::vector<i64> sA, const std::vector<i64> &oA, int c_buf, std::vector<i64> sC,
              const std::vector<i64> &oC, double alpha, double beta) {
        SigmaStep s{};
        s.name = cur;
        s.kind = STEP_PERM;
        s.p.nd = (int)dims.size();
        s.p.total = 1;
        for (int d = 0; d < s.p.nd; ++d) {
            s.p.dims[d] = dims[d];
            s.p.sA[d] = sA[d];
            s.p.sC[d] = sC[d];
            s.p.total *= dims[d];
        }
        s.p.batch = (int)oC.size();
        s.p.alpha = make_double2(alpha, 0.0);
        s.p.beta = make_double2(beta, 0.0);
        s.a_buf = BUF_SCRATCH;
        s.c_buf = c_buf;
        s.offA_pos = push(oA);
        s.offC_pos = push(oC);
        P->steps.push_back(s);
    }
    void fov(int kind) {
        SigmaStep s{};
        s.name = kind == STEP_FOV_IP ? "ip_fov" : "ea_fov";
        s.kind = kind;
        P->steps.push_back(s);
    }
};

enum { SEG_X = 0, SEG_R, SEG_Q, SEG_T1, SEG_T3, SEG_XT, SEG_SMALL, SEG_D0, SEG_D1, SEG_SPLITK, SEG_END };

// Scratch segments (complex elements) of a plan with nv columns. D0 / D1 hold the intermediates of
// the EA terms formed from the density-fitting factors (sized only when a plan uses them):
//   D0 = X0 [nk][Q][v][nv] | X1 [nk][Q][o][nv] | y2 [o][nv] | Zc [nk][Q][v][nv]
//   D1 = Y [nk][nk][o][o][o][nv]  or  Zx [nk][nk][Q][v][nv]
void scratch_layout(const ccgf_handle *h, int nv, i64 seg[SEG_END + 1], bool df_terms) {
    const i64 nk = h->nk, nk2 = (i64)h->nk * h->nk, o = h->o, v = h->v, Q = h->naux;
    i64 dmax = h->dim_ip > h->dim_ea ? h->dim_ip : h->dim_ea;
    i64 r2max = nk2 * o * v * (o > v ? o : v);
    const i64 d0 = df_terms ? (2 * nk * Q * v + nk * Q * o + o) * nv : 0;
    const i64 d1 = df_terms ? std::max(nk2 * o * o * o, nk2 * Q * v) * nv : 0;
    // split-K partials of the launcher's own splits: at most 304 slices of an (o+v) x nv product
    // (the autotuner's wave-filling splits use a separate workspace of the handle)
    i64 sizes[SEG_END] = {dmax * nv, r2max * nv, r2max * nv, r2max * nv, r2max * nv, r2max * nv, (o + v) * (i64)nv, d0, d1,
                          304 * (o + v) * (i64)nv};
    i64 pos = 0;
    for (int s = 0; s < SEG_END; ++s) {
        seg[s] = pos;
        pos += (sizes[s] + 31) / 32 * 32;
    }
    seg[SEG_END] = pos;
}

// offsets of the pieces of segment D0 (see scratch_layout)
struct D0Parts {
    i64 x0, x1, y2, zc;
};
D0Parts d0_parts(const ccgf_handle *h, const SigmaPlan *P) {
    const i64 nk = h->nk, o = h->o, v = h->v, Q = h->naux, NV = P->nv, b = P->seg[SEG_D0];
    return D0Parts{b, b + nk * Q * v * NV, b + nk * Q * v * NV + nk * Q * o * NV, b + nk * Q * v * NV + nk * Q * o * NV + o * NV};
}

// The EA r1 -> r2 coupling, sum_e W_vvvo[ka,kb,K][a,b,e,j] r1[e], evaluated from the density-fitting
// factors (e at K, kb = K + kj - ka); W_vvvo = <ab|ej> + sum <mn|ej> t_mn^ab - sum Fov[me] t_mj^ab
//   - sum <mb|ef> t_mj^af + sum (2<ma|fe> - <ma|ef>) t_mj^fb - sum <ma|fe> t_mj^bf, with <pq|rs> = (pr|qs):
//   X0[ka][Q][a] = sum_e L~[ka,K,Q][a,e] r_e,  X1[km][Q][m] = sum_e L~[km,K,Q][m,e] r_e,  y2[m] = Fov[K] r
//   T0  s2 += sum_Q X0[ka][Q][a] L~[kb,kj,Q][b,j]                                     (first write of s2)
//   T1  Y[kj][km][m,n,j] = sum_Q X1[km][Q][m] L~[kn,kj,Q][n,j]  (kn = K + kj - km)
//       s2 += sum_{km,m,n} t[km,kn,ka][m,n,a,b] Y[kj][km][m,n,j]    (after `extra_y` adds to Y)
//   T2  s2 -= sum_m t[K,kj,ka][m,j,a,b] y2[m]
//   T3  Y3[km][kb][m,b,f] = sum_Q X1[km][Q][m] L~[kb,kf,Q][b,f]  (kf = km + kb - K)
//       s2 -= sum_{km,m,f} t[km,kj,ka][m,j,a,f] Y3[km][kb][m,b,f]
//   T4  ZA[km][ka][m,a,f] = sum_Q L~[km,kf,Q][m,f] X0[ka][Q][a],  ZB = 2 ZA - sum_Q X1[km][Q][m] L~[ka,kf,Q][a,f]
//       (kf = km + ka - K);  s2 += sum_{km,m,f} ZB[km][ka][m,a,f] t[km,kj,kf][m,j,f,b]
//   T5  s2 -= sum_{km,m,f} ZA[km][ka][m,a,f] t[km,kj,kb][m,j,b,f]
template <typename Extra>
void emit_ea_r1_terms(PlanBuilder &B, const ccgf_handle *h, SigmaPlan *P, int K, Extra extra_y) {
    const auto &km = h->km;
    const int nk = h->nk, o = h->o, v = h->v, n = h->n, Q = h->naux;
    const i64 NV = P->nv, S2 = (i64)o * v * v, v2 = (i64)v * v, o2 = (i64)o * o, n2 = (i64)n * n;
    const i64 sx = P->seg[SEG_X];
    const D0Parts d0 = d0_parts(h, P);
    auto row = [&](int kj, int ka) -> i64 { return v + ((i64)kj * nk + ka) * S2; };
    auto LB = [&](int k1, int k2) -> i64 { return ((i64)k1 * nk + k2) * Q * n2; };
    auto TB = [&](int ki, int kj, int ka) -> i64 { return (((i64)ki * nk + kj) * nk + ka) * o2 * v2; };
    const IMap one = imap_single(1);
    B.cur = "ea_s2_r1_df";
    {
        std::vector<i64> a0, a1, bx, c0, c1;
        for (int k = 0; k < nk; ++k) {
            a0.push_back(LB(k, K) + (i64)o * n + o);
            a1.push_back(LB(k, K) + o);
            bx.push_back(sx);
            c0.push_back(d0.x0 + (i64)k * Q * v * NV);
            c1.push_back(d0.x1 + (i64)k * Q * o * NV);
        }
        // X0: rows (Q, a), X1: rows (Q, m); contraction e; columns = the nv vectors
        B.tgemm(Q * v, (int)NV, v, 1, BUF_LD, imap_pair(v, n2, n), one, a0, BUF_SCRATCH, imap_single(NV), one, bx, BUF_SCRATCH,
                imap_single(NV), one, c0, 1.0, 0.0);
        B.tgemm(Q * o, (int)NV, v, 1, BUF_LD, imap_pair(o, n2, n), one, a1, BUF_SCRATCH, imap_single(NV), one, bx, BUF_SCRATCH,
                imap_single(NV), one, c1, 1.0, 0.0);
        B.gemm(o, (int)NV, v, 1, BUF_FOV, v, 1, {(i64)K * o * v}, NV, 1, {sx}, BUF_SCRATCH, NV, 1, {d0.y2}, 1.0, 0.0);
    }
    // T0 (first write of every s2 block): rows (a, c), columns (b, j), contraction Q
    {
        std::vector<i64> oA, oB, oC;
        for (int kj = 0; kj < nk; ++kj)
            for (int ka = 0; ka < nk; ++ka) {
                const int kb = km.c(K, ka, kj);
                oA.push_back(d0.x0 + (i64)ka * Q * v * NV);
                oB.push_back(LB(kb, kj) + (i64)o * n);
                oC.push_back(row(kj, ka) * NV);
            }
        B.tgemm(v * (int)NV, v * o, Q, 1, BUF_SCRATCH, imap_single(1), imap_single(v * NV), oA, BUF_LD, imap_single(n2),
                imap_pair(o, n, 1), oB, BUF_Y, imap_pair((int)NV, v * NV, 1), imap_pair(o, NV, v2 * NV), oC, 1.0, 0.0);
    }
    // T1: Y[kj][km][m][n][j][c] in D1, rows (m, c), columns (n, j), contraction Q
    {
        std::vector<i64> oA, oB, oC;
        for (int kj = 0; kj < nk; ++kj)
            for (int kmm = 0; kmm < nk; ++kmm) {
                const int kn = km.c(K, kmm, kj);
                oA.push_back(d0.x1 + (i64)kmm * Q * o * NV);
                oB.push_back(LB(kn, kj));
                oC.push_back(P->seg[SEG_D1] + ((i64)kj * nk + kmm) * o2 * o * NV);
            }
        B.tgemm(o * (int)NV, (int)o2, Q, 1, BUF_SCRATCH, imap_single(1), imap_single(o * NV), oA, BUF_LD, imap_single(n2),
                imap_pair(o, n, 1), oB, BUF_SCRATCH, imap_pair((int)NV, o2 * NV, 1), imap_pair(o, o * NV, NV), oC, 1.0, 0.0);
    }
    extra_y();
    // s2 += sum_{km,m,n} t[km,kn,ka][m,n,a,b] Y[kj][km][m,n,j]: rows (a, b), columns (j, c), contraction (m, n)
    {
        std::vector<i64> oA, oB, oC;
        for (int kj = 0; kj < nk; ++kj)
            for (int ka = 0; ka < nk; ++ka) {
                for (int kmm = 0; kmm < nk; ++kmm) {
                    const int kn = km.c(K, kmm, kj);
                    oA.push_back(TB(kmm, kn, ka));
                    oB.push_back(P->seg[SEG_D1] + ((i64)kj * nk + kmm) * o2 * o * NV);
                }
                oC.push_back(row(kj, ka) * NV);
            }
        B.tgemm((int)v2, o * (int)NV, (int)o2, nk, BUF_T2, one, imap_pair(o, o * v2, v2), oA, BUF_SCRATCH,
                imap_pair(o, o2 * NV, o * NV), imap_pair((int)NV, NV, 1), oB, BUF_Y, imap_single(NV), imap_pair((int)NV, v2 * NV, 1),
                oC, 1.0, 1.0);
    }
    // T2: s2 -= t[K,kj,ka][m,j,a,b] y2[m]
    {
        std::vector<i64> oA, oB, oC;
        for (int kj = 0; kj < nk; ++kj)
            for (int ka = 0; ka < nk; ++ka) {
                oA.push_back((((i64)K * nk + kj) * nk + ka) * S2 * o);
                oB.push_back(d0.y2);
                oC.push_back(row(kj, ka) * NV);
            }
        B.gemm((int)S2, (int)NV, o, 1, BUF_T2EA, o, 1, oA, NV, 1, oB, BUF_Y, NV, 1, oC, -1.0, 1.0);
    }
    // T3: Y3[km][kb][m][b][f][c] in R, rows (m, c), columns (b, f), contraction Q
    {
        std::vector<i64> oA, oB, oC;
        for (int kmm = 0; kmm < nk; ++kmm)
            for (int kb = 0; kb < nk; ++kb) {
                const int kf = km.c(kmm, K, kb);
                oA.push_back(d0.x1 + (i64)kmm * Q * o * NV);
                oB.push_back(LB(kb, kf) + (i64)o * n + o);
                oC.push_back(P->seg[SEG_R] + ((i64)kmm * nk + kb) * S2 * NV);
            }
        B.tgemm(o * (int)NV, (int)v2, Q, 1, BUF_SCRATCH, imap_single(1), imap_single(o * NV), oA, BUF_LD, imap_single(n2),
                imap_pair(v, n, 1), oB, BUF_SCRATCH, imap_pair((int)NV, v2 * NV, 1), imap_pair(v, v * NV, NV), oC, 1.0, 0.0);
    }
    // s2 -= sum_{km,m,f} t[km,kj,ka][m,j,a,f] Y3[km][kb][m,b,f]: rows (j, a), columns (b, c), contraction (m, f)
    {
        std::vector<i64> oA, oB, oC;
        for (int kj = 0; kj < nk; ++kj)
            for (int ka = 0; ka < nk; ++ka) {
                const int kb = km.c(K, ka, kj);
                for (int kmm = 0; kmm < nk; ++kmm) {
                    oA.push_back(TB(kmm, kj, ka));
                    oB.push_back(P->seg[SEG_R] + ((i64)kmm * nk + kb) * S2 * NV);
                }
                oC.push_back(row(kj, ka) * NV);
            }
        B.tgemm(o * v, v * (int)NV, o * v, nk, BUF_T2, imap_pair(v, v2, v), imap_pair(v, o * v2, 1), oA, BUF_SCRATCH,
                imap_pair(v, v2 * NV, NV), imap_pair((int)NV, v * NV, 1), oB, BUF_Y, imap_pair(v, v2 * NV, v * NV),
                imap_pair((int)NV, NV, 1), oC, -1.0, 1.0);
    }
    // T4 / T5: ZA[km][ka][m][a][f][c] in Q, ZB = 2 ZA - (X1 . L~) in T1; rows (m, f) or (m, c)
    {
        std::vector<i64> aL, bX, cA, cB, aX, bL;
        for (int kmm = 0; kmm < nk; ++kmm)
            for (int ka = 0; ka < nk; ++ka) {
                const int kf = km.c(kmm, K, ka);
                aL.push_back(LB(kmm, kf) + o);
                bX.push_back(d0.x0 + (i64)ka * Q * v * NV);
                cA.push_back(P->seg[SEG_Q] + ((i64)kmm * nk + ka) * S2 * NV);
                cB.push_back(P->seg[SEG_T1] + ((i64)kmm * nk + ka) * S2 * NV);
                aX.push_back(d0.x1 + (i64)kmm * Q * o * NV);
                bL.push_back(LB(ka, kf) + (i64)o * n + o);
            }
        const IMap cm_mf = imap_pair(v, v2 * NV, NV), cn_ac = imap_pair((int)NV, v * NV, 1);
        B.tgemm(o * v, v * (int)NV, Q, 1, BUF_LD, imap_pair(v, n, 1), imap_single(n2), aL, BUF_SCRATCH, imap_single(v * NV),
                imap_single(1), bX, BUF_SCRATCH, cm_mf, cn_ac, cA, 1.0, 0.0);
        B.tgemm(o * v, v * (int)NV, Q, 1, BUF_LD, imap_pair(v, n, 1), imap_single(n2), aL, BUF_SCRATCH, imap_single(v * NV),
                imap_single(1), bX, BUF_SCRATCH, cm_mf, cn_ac, cB, 2.0, 0.0);
        // - sum_Q X1[km][Q][m][c] L~[ka,kf,Q][a,f]: rows (m, c), columns (a, f)
        B.tgemm(o * (int)NV, (int)v2, Q, 1, BUF_SCRATCH, imap_single(1), imap_single(o * NV), aX, BUF_LD, imap_single(n2),
                imap_pair(v, n, 1), bL, BUF_SCRATCH, imap_pair((int)NV, v2 * NV, 1), imap_pair(v, v * NV, NV), cB, -1.0, 1.0);
    }
    {
        std::vector<i64> a4, a5, bB, bA, oC;
        for (int kj = 0; kj < nk; ++kj)
            for (int ka = 0; ka < nk; ++ka) {
                const int kb = km.c(K, ka, kj);
                for (int kmm = 0; kmm < nk; ++kmm) {
                    const int kf = km.c(kmm, K, ka);
                    a4.push_back(TB(kmm, kj, kf));   // t[km,kj,kf][m,j,f,b]
                    a5.push_back(TB(kmm, kj, kb));   // t[km,kj,kb][m,j,b,f]
                    bB.push_back(P->seg[SEG_T1] + ((i64)kmm * nk + ka) * S2 * NV);
                    bA.push_back(P->seg[SEG_Q] + ((i64)kmm * nk + ka) * S2 * NV);
                }
                oC.push_back(row(kj, ka) * NV);
            }
        // rows (j, b), columns (a, c), contraction (m, f)
        const IMap bk_mf = imap_pair(v, v2 * NV, NV), bn_ac = imap_pair((int)NV, v * NV, 1);
        const IMap cm_jb = imap_pair(v, v2 * NV, NV), cn_ac = imap_pair((int)NV, v * NV, 1);
        B.tgemm(o * v, v * (int)NV, o * v, nk, BUF_T2, imap_pair(v, v2, 1), imap_pair(v, o * v2, v), a4, BUF_SCRATCH, bk_mf, bn_ac,
                bB, BUF_Y, cm_jb, cn_ac, oC, 1.0, 1.0);
        B.tgemm(o * v, v * (int)NV, o * v, nk, BUF_T2, imap_pair(v, v2, v), imap_pair(v, o * v2, 1), a5, BUF_SCRATCH, bk_mf, bn_ac,
                bA, BUF_Y, cm_jb, cn_ac, oC, -1.0, 1.0);
    }
}

SigmaPlan *build_plan_ea(const ccgf_handle *h, int K, int nv, bool r1_only = false) {
    const auto &km = h->km;
    const int nk = h->nk, o = h->o, v = h->v;
    SigmaPlan *P = new SigmaPlan();
    P->sector = CCGF_SECTOR_EA;
    P->K = K;
    P->nv = nv;
    scratch_layout(h, nv, P->seg, h->direct || r1_only);
    P->scratch_elems = P->seg[SEG_END];
    PlanBuilder B{P, {}};
    const i64 S2 = (i64)o * v * v, NV = nv;
    const i64 sx = P->seg[SEG_X];
    auto row = [&](int kj, int ka) -> i64 { return v + ((i64)kj * nk + ka) * S2; };
    const i64 v2 = (i64)v * v, ov = (i64)o * v, nk2 = (i64)nk * nk;

    const int n = h->n, Q = h->naux;
    const i64 n2 = (i64)n * n, o2 = (i64)o * o;
    auto LB = [&](int k1, int k2) -> i64 { return ((i64)k1 * nk + k2) * Q * n2; };
    if (r1_only) {
        // the r1 -> r2 coupling alone (applied to unit vectors it gives the stored W_vvvo[K])
        emit_ea_r1_terms(B, h, P, K, [] {});
        P->host_off = B.off;
        return P;
    }

    // s1[a] = Fvv[K] r1 (first write)
    B.cur = "ea_s1_fvv";
    B.gemm(v, nv, v, 1, BUF_FVV, v, 1, {(i64)K * v2}, NV, 1, {sx}, BUF_Y, NV, 1, {0}, 1.0, 0.0);
    B.fov(STEP_FOV_EA);
    // s1 += sum (2<am|ef> - <am|fe>) r2[km,ke][m,e,f],  <a K m km|e ke f kf> = (a e|m f), kf = K + km - ke
    B.cur = "ea_s1_vovv";
    if (!h->direct) {
        B.gemm(v, nv, (int)(nk2 * o * v2), 1, BUF_UVOVV, nk2 * o * v2, 1, {(i64)K * v * nk2 * o * v2}, NV, 1, {sx + v * NV},
               BUF_Y, NV, 1, {0}, 1.0, 1.0);
    } else {
        // Coulomb: Zc[ke][Q][e] = sum_{km,m,f} L~[km,kf,Q][m,f] r2[km,ke][m,e,f];  s1 += 2 sum L~[K,ke,Q][a,e] Zc[ke][Q][e]
        // exchange: Zx[km][ke][Q][f] = sum_{m,e} L~[km,ke,Q][m,e] r2[km,ke][m,e,f];  s1 -= sum L~[K,kf,Q][a,f] Zx[km][ke][Q][f]
        const D0Parts d0 = d0_parts(h, P);
        std::vector<i64> zA, zB, zC, sA, sB, xA, xB, xC, tA, tB;
        for (int ke = 0; ke < nk; ++ke) {
            for (int kmm = 0; kmm < nk; ++kmm) {
                const int kf = km.c(K, ke, kmm);
                zA.push_back(LB(kmm, kf) + o);
                zB.push_back(sx + row(kmm, ke) * NV);
            }
            zC.push_back(d0.zc + (i64)ke * Q * v * NV);
            sA.push_back(LB(K, ke) + (i64)o * n + o);
            sB.push_back(d0.zc + (i64)ke * Q * v * NV);
        }
        for (int kmm = 0; kmm < nk; ++kmm)
            for (int ke = 0; ke < nk; ++ke) {
                const int kf = km.c(K, ke, kmm);
                xA.push_back(LB(kmm, ke) + o);
                xB.push_back(sx + row(kmm, ke) * NV);
                xC.push_back(P->seg[SEG_D1] + ((i64)kmm * nk + ke) * Q * v * NV);
                tA.push_back(LB(K, kf) + (i64)o * n + o);
                tB.push_back(P->seg[SEG_D1] + ((i64)kmm * nk + ke) * Q * v * NV);
            }
        // Zc: rows Q, columns (e, c), contraction (m, f) over km
        B.tgemm(Q, v * nv, (int)ov, nk, BUF_LD, imap_single(n2), imap_pair(v, n, 1), zA, BUF_SCRATCH, imap_pair(v, v2 * NV, NV),
                imap_pair(nv, v * NV, 1), zB, BUF_SCRATCH, imap_single(v * NV), imap_single(1), zC, 1.0, 0.0);
        // s1 += 2 sum_{ke} L~[K,ke][a,(Q,e)] Zc[ke][(Q,e)][c]
        B.tgemm(v, nv, Q * v, nk, BUF_LD, imap_single(n), imap_pair(v, n2, 1), sA, BUF_SCRATCH, imap_pair(v, v * NV, NV),
                imap_single(1), sB, BUF_Y, imap_single(NV), imap_single(1), {0}, 2.0, 1.0);
        // Zx: rows Q, columns (f, c), contraction (m, e)
        B.tgemm(Q, v * nv, (int)ov, 1, BUF_LD, imap_single(n2), imap_pair(v, n, 1), xA, BUF_SCRATCH, imap_pair(v, v2 * NV, v * NV),
                imap_single(1), xB, BUF_SCRATCH, imap_single(v * NV), imap_single(1), xC, 1.0, 0.0);
        // s1 -= sum_{km,ke} L~[K,kf][a,(Q,f)] Zx[km][ke][(Q,f)][c]
        B.tgemm(v, nv, Q * v, nk * nk, BUF_LD, imap_single(n), imap_pair(v, n2, 1), tA, BUF_SCRATCH, imap_pair(v, v * NV, NV),
                imap_single(1), tB, BUF_Y, imap_single(NV), imap_single(1), {0}, -1.0, 1.0);
    }
    // s2 = Wvvvo r1 (first write of every block)
    B.cur = "ea_s2_wvvvo";
    if (!h->direct) {
        // stored W_vvvo[K] as rows (kj, ka, j, a, b) of the r2 part, columns e
        B.gemm((int)(nk2 * o * v2), nv, v, 1, BUF_WVVVO, v, 1, {(i64)K * nk2 * o * v2 * v}, NV, 1, {sx}, BUF_Y, NV, 1, {v * NV},
               1.0, 0.0);
    } else {
        // from the density-fitting factors; the T2 part of the ladder, sum_{ke,e,f} <mn|ef> r2[kj,ke][j,e,f]
        // = sum (m e|n f) r2 (kn = K + kj - km), joins the Y of the T1 term (both are contracted with t[km,kn,ka])
        emit_ea_r1_terms(B, h, P, K, [&] {
            B.cur = "ea_ladder_t2_df";
            std::vector<i64> oA, oB, oC;
            for (int kj = 0; kj < nk; ++kj)
                for (int kmm = 0; kmm < nk; ++kmm) {
                    const int kn = km.c(K, kmm, kj);
                    for (int ke = 0; ke < nk; ++ke) {
                        oA.push_back((((i64)kmm * nk + ke) * nk + kn) * o2 * v2);
                        oB.push_back(sx + row(kj, ke) * NV);
                    }
                    oC.push_back(P->seg[SEG_D1] + ((i64)kj * nk + kmm) * o2 * o * NV);
                }
            // rows (m, n), columns (j, c), contraction (e, f)
            B.tgemm((int)o2, o * nv, (int)v2, nk, BUF_OVOV, imap_pair(o, v * o * v, v), imap_pair(v, ov, 1), oA, BUF_SCRATCH,
                    imap_pair(v, v * NV, NV), imap_pair(nv, v2 * NV, 1), oB, BUF_SCRATCH, imap_pair(o, o2 * NV, o * NV),
                    imap_pair(nv, NV, 1), oC, 1.0, 1.0);
            B.cur = "ea_s2_r1_df";
        });
    }
    // s2 += Fvv[ka](a,e) r2[j,e,b]
    B.cur = "ea_s2_fvv_a";
    {
        std::vector<i64> oA, oB, oC;
        for (int kj = 0; kj < nk; ++kj)
            for (int ka = 0; ka < nk; ++ka)
                for (int j = 0; j < o; ++j) {
                    oA.push_back((i64)ka * v2);
                    oB.push_back(sx + (row(kj, ka) + j * v2) * NV);
                    oC.push_back((row(kj, ka) + j * v2) * NV);
                }
        B.gemm(v, (int)(v * NV), v, 1, BUF_FVV, v, 1, oA, v * NV, 1, oB, BUF_Y, v * NV, 1, oC, 1.0, 1.0);
    }
    // s2 += Fvv[kb](b,e) r2[j,a,e]
    B.cur = "ea_s2_fvv_b";
    {
        std::vector<i64> oA, oB, oC;
        for (int kj = 0; kj < nk; ++kj)
            for (int ka = 0; ka < nk; ++ka) {
                int kb = km.c(K, ka, kj);
                for (int j = 0; j < o; ++j)
                    for (int a = 0; a < v; ++a) {
                        i64 r = row(kj, ka) + (j * v + a) * (i64)v;
                        oA.push_back((i64)kb * v2);
                        oB.push_back(sx + r * NV);
                        oC.push_back(r * NV);
                    }
            }
        B.gemm(v, nv, v, 1, BUF_FVV, v, 1, oA, NV, 1, oB, BUF_Y, NV, 1, oC, 1.0, 1.0);
    }
    // s2 -= Foo[kj](m,j) r2[m,a,b]
    B.cur = "ea_s2_foo";
    {
        std::vector<i64> oA, oB, oC;
        for (int kj = 0; kj < nk; ++kj)
            for (int ka = 0; ka < nk; ++ka) {
                oA.push_back((i64)kj * o * o);
                oB.push_back(sx + row(kj, ka) * NV);
                oC.push_back(row(kj, ka) * NV);
            }
        B.gemm(o, (int)(v2 * NV), o, 1, BUF_FOO, 1, o, oA, v2 * NV, 1, oB, BUF_Y, v2 * NV, 1, oC, -1.0, 1.0);
    }
    // R'[ka][km][m][e][a] = r2[km,ka][m,a,e]
    B.cur = "ea_ring_gather";
    {
        std::vector<i64> oA, oC;
        for (int ka = 0; ka < nk; ++ka)
            for (int kmm = 0; kmm < nk; ++kmm) {
                oA.push_back(sx + row(kmm, ka) * NV);
                oC.push_back(P->seg[SEG_R] + ((i64)ka * nk + kmm) * S2 * NV);
            }
        B.perm({o, v, v, NV}, {v2 * NV, NV, v * NV, 1}, oA, BUF_SCRATCH, {v2 * NV, v * NV, NV, 1}, oC, 1.0, 0.0);
    }
    // ring: T1[kj][ka][j][b][a] = sum_km W1[kb][kj][km] R'[ka][km] + W2[kb][kj][km] Q'[ka][km], Q' = r2[km,ke][m,e,a]
    B.cur = "ea_ring_w1w2";
    {
        std::vector<i64> oA, oB, oC;
        const i64 blk = ov * ov;
        for (int kj = 0; kj < nk; ++kj)
            for (int ka = 0; ka < nk; ++ka) {
                int kb = km.c(K, ka, kj);
                for (int kmm = 0; kmm < nk; ++kmm) {
                    int ke = km.c(K, ka, kmm);
                    oA.push_back(0 * h->wov_seg + (((i64)kb * nk + kj) * nk + kmm) * blk);
                    oB.push_back(P->seg[SEG_R] + ((i64)ka * nk + kmm) * S2 * NV);
                    oA.push_back(1 * h->wov_seg + (((i64)kb * nk + kj) * nk + kmm) * blk);
                    oB.push_back(sx + row(kmm, ke) * NV);
                }
                oC.push_back(P->seg[SEG_T1] + ((i64)kj * nk + ka) * S2 * NV);
            }
        B.gemm((int)ov, (int)(v * NV), (int)ov, 2 * nk, BUF_WOV3, ov, 1, oA, v * NV, 1, oB, BUF_SCRATCH, v * NV, 1, oC, 1.0,
               0.0);
        std::vector<i64> pA, pC;
        for (int kj = 0; kj < nk; ++kj)
            for (int ka = 0; ka < nk; ++ka) {
                pA.push_back(P->seg[SEG_T1] + ((i64)kj * nk + ka) * S2 * NV);
                pC.push_back(row(kj, ka) * NV);
            }
        B.perm({o, v, v, NV}, {v2 * NV, v * NV, NV, 1}, pA, BUF_Y, {v2 * NV, NV, v * NV, 1}, pC, 1.0, 1.0);
    }
    // ring: s2[j,a,b] += sum_km WN[ka][kj][km](j,a;m,e) r2[km,ke2][m,e,b], ke2 = km + ka - kj
    B.cur = "ea_ring_wn";
    {
        std::vector<i64> oA, oB, oC;
        const i64 blk = ov * ov;
        for (int kj = 0; kj < nk; ++kj)
            for (int ka = 0; ka < nk; ++ka) {
                for (int kmm = 0; kmm < nk; ++kmm) {
                    int ke2 = km.c(kmm, kj, ka);
                    oA.push_back(2 * h->wov_seg + (((i64)ka * nk + kj) * nk + kmm) * blk);
                    oB.push_back(sx + row(kmm, ke2) * NV);
                }
                oC.push_back(row(kj, ka) * NV);
            }
        B.gemm((int)ov, (int)(v * NV), (int)ov, nk, BUF_WOV3, ov, 1, oA, v * NV, 1, oB, BUF_Y, v * NV, 1, oC, 1.0, 1.0);
    }
    // ladder (pair-symmetric): R+/- on pair representatives of every pair momentum s = K + kj,
    // S+/- = W+/-[s] R+/-[s], then S(alpha) = S+ + S-, S(Pi alpha) = S+ - S- scattered into s2
    B.cur = "ea_ladder_wvvvv";
    {
        const int Pp = h->lad_Pp, Pm = h->lad_Pm;
        const i64 on = (i64)o * NV;
        SigmaStep g{};
        g.name = B.cur;
        g.kind = STEP_LADDER_GATHER;
        g.lad_rp = P->seg[SEG_XT];
        g.lad_rm = P->seg[SEG_R];
        P->steps.push_back(g);
        std::vector<i64> aP, bP, cP, aM, bM, cM;
        for (int sp = 0; sp < nk; ++sp) {
            aP.push_back((i64)sp * Pp * Pp);
            bP.push_back(P->seg[SEG_XT] + (i64)sp * Pp * on);
            cP.push_back(P->seg[SEG_T3] + (i64)sp * Pp * on);
            aM.push_back((i64)sp * Pm * Pm);
            bM.push_back(P->seg[SEG_R] + (i64)sp * Pm * on);
            cM.push_back(P->seg[SEG_T1] + (i64)sp * Pm * on);
        }
        B.gemm(Pp, (int)on, Pp, 1, BUF_WPLUS, Pp, 1, aP, on, 1, bP, BUF_SCRATCH, on, 1, cP, 1.0, 0.0);
        B.gemm(Pm, (int)on, Pm, 1, BUF_WMINUS, Pm, 1, aM, on, 1, bM, BUF_SCRATCH, on, 1, cM, 1.0, 0.0);
        SigmaStep sc{};
        sc.name = B.cur;
        sc.kind = STEP_LADDER_SCATTER;
        sc.lad_rp = P->seg[SEG_T3];
        sc.lad_rm = P->seg[SEG_T1];
        P->steps.push_back(sc);
    }
    // three-body: Ysm[m] = sum (2<mn|ef> - <mn|fe>) r2[kn,ke][n,e,f];  s2 -= t2[K,kj,ka][m,j,a,b] Ysm[m]
    B.cur = "ea_threebody";
    {
        const i64 sm = P->seg[SEG_SMALL];
        B.gemm(o, nv, (int)(nk2 * o * v2), 1, BUF_UOOVV_EA, nk2 * o * v2, 1, {(i64)K * o * nk2 * o * v2}, NV, 1,
               {sx + v * NV}, BUF_SCRATCH, NV, 1, {sm}, 1.0, 0.0);
        std::vector<i64> oA, oB, oC;
        for (int kj = 0; kj < nk; ++kj)
            for (int ka = 0; ka < nk; ++ka) {
                oA.push_back((((i64)K * nk + kj) * nk + ka) * S2 * o);
                oB.push_back(sm);
                oC.push_back(row(kj, ka) * NV);
            }
        B.gemm((int)S2, nv, o, 1, BUF_T2EA, o, 1, oA, NV, 1, oB, BUF_Y, NV, 1, oC, -1.0, 1.0);
    }
    P->host_off = B.off;
    return P;
}

SigmaPlan *build_plan_ip(const ccgf_handle *h, int K, int nv) {
    const auto &km = h->km;
    const int nk = h->nk, o = h->o, v = h->v;
    SigmaPlan *P = new SigmaPlan();
    P->sector = CCGF_SECTOR_IP;
    P->K = K;
    P->nv = nv;
    scratch_layout(h, nv, P->seg, false);
    P->scratch_elems = P->seg[SEG_END];
    PlanBuilder B{P, {}};
    const i64 S2 = (i64)o * o * v, NV = nv;
    const i64 sx = P->seg[SEG_X];
    auto row = [&](int ki, int kj) -> i64 { return o + ((i64)ki * nk + kj) * S2; };
    const i64 o2 = (i64)o * o, ov = (i64)o * v, nk2 = (i64)nk * nk;

    // s1 = -Foo[K]^T r1
    B.cur = "ip_s1_foo";
    B.gemm(o, nv, o, 1, BUF_FOO, 1, o, {(i64)K * o2}, NV, 1, {sx}, BUF_Y, NV, 1, {0}, -1.0, 0.0);
    B.fov(STEP_FOV_IP);
    // s1 -= sum (2<mn|ie> - <mn|ei>) r2
    B.cur = "ip_s1_ooov";
    B.gemm(o, nv, (int)(nk2 * S2), 1, BUF_UOOOV, nk2 * S2, 1, {(i64)K * o * nk2 * S2}, NV, 1, {sx + o * NV}, BUF_Y, NV, 1,
           {0}, -1.0, 1.0);
    // s2 = -Wovoo r1 (first write)
    B.cur = "ip_s2_wovoo";
    {
        std::vector<i64> oA, oB, oC;
        for (int ki = 0; ki < nk; ++ki)
            for (int kj = 0; kj < nk; ++kj) {
                oA.push_back((((i64)K * nk + ki) * nk + kj) * S2 * o);
                oB.push_back(sx);
                oC.push_back(row(ki, kj) * NV);
            }
        B.gemm((int)S2, nv, o, 1, BUF_WOVOO, o, 1, oA, NV, 1, oB, BUF_Y, NV, 1, oC, -1.0, 0.0);
    }
    // s2 += Fvv[ka](a,e) r2[i,j,e]
    B.cur = "ip_s2_fvv";
    {
        std::vector<i64> oA, oB, oC;
        for (int ki = 0; ki < nk; ++ki)
            for (int kj = 0; kj < nk; ++kj) {
                int ka = km.c(ki, K, kj);
                for (int ij = 0; ij < o * o; ++ij) {
                    i64 r = row(ki, kj) + (i64)ij * v;
                    oA.push_back((i64)ka * v * v);
                    oB.push_back(sx + r * NV);
                    oC.push_back(r * NV);
                }
            }
        B.gemm(v, nv, v, 1, BUF_FVV, v, 1, oA, NV, 1, oB, BUF_Y, NV, 1, oC, 1.0, 1.0);
    }
    // s2 -= Foo[ki](m,i) r2[m,j,a]
    B.cur = "ip_s2_foo_i";
    {
        std::vector<i64> oA, oB, oC;
        for (int ki = 0; ki < nk; ++ki)
            for (int kj = 0; kj < nk; ++kj) {
                oA.push_back((i64)ki * o2);
                oB.push_back(sx + row(ki, kj) * NV);
                oC.push_back(row(ki, kj) * NV);
            }
        B.gemm(o, (int)(ov * NV), o, 1, BUF_FOO, 1, o, oA, ov * NV, 1, oB, BUF_Y, ov * NV, 1, oC, -1.0, 1.0);
    }
    // s2 -= Foo[kj](m,j) r2[i,m,a]
    B.cur = "ip_s2_foo_j";
    {
        std::vector<i64> oA, oB, oC;
        for (int ki = 0; ki < nk; ++ki)
            for (int kj = 0; kj < nk; ++kj)
                for (int i = 0; i < o; ++i) {
                    oA.push_back((i64)kj * o2);
                    oB.push_back(sx + (row(ki, kj) + i * ov) * NV);
                    oC.push_back((row(ki, kj) + i * ov) * NV);
                }
        B.gemm(o, (int)(v * NV), o, 1, BUF_FOO, 1, o, oA, v * NV, 1, oB, BUF_Y, v * NV, 1, oC, -1.0, 1.0);
    }
    // s2 += sum_km Woooo[ki][kj](i,j;km,m,n) r2[km,kn][m,n,a]
    B.cur = "ip_ladder_woooo";
    {
        std::vector<i64> oA, oB, oC;
        for (int ki = 0; ki < nk; ++ki)
            for (int kj = 0; kj < nk; ++kj) {
                for (int kmm = 0; kmm < nk; ++kmm) {
                    int kn = km.c(ki, kmm, kj);
                    oA.push_back(((i64)ki * nk + kj) * o2 * nk * o2 + (i64)kmm * o2);
                    oB.push_back(sx + row(kmm, kn) * NV);
                }
                oC.push_back(row(ki, kj) * NV);
            }
        B.gemm((int)o2, (int)(v * NV), (int)o2, nk, BUF_WOOOO, nk * o2, 1, oA, v * NV, 1, oB, BUF_Y, v * NV, 1, oC, 1.0, 1.0);
    }
    // R'[ki][km][m][e][i] = r2[ki,km][i,m,e];  Q'[kj][km][m][e][j] = r2[km,kj][m,j,e]
    B.cur = "ip_ring_gather";
    {
        std::vector<i64> oA, oC;
        for (int ki = 0; ki < nk; ++ki)
            for (int kmm = 0; kmm < nk; ++kmm) {
                oA.push_back(sx + row(ki, kmm) * NV);
                oC.push_back(P->seg[SEG_R] + ((i64)ki * nk + kmm) * S2 * NV);
            }
        B.perm({o, v, o, NV}, {v * NV, NV, ov * NV, 1}, oA, BUF_SCRATCH, {v * o * NV, o * NV, NV, 1}, oC, 1.0, 0.0);
        std::vector<i64> qA, qC;
        for (int kj = 0; kj < nk; ++kj)
            for (int kmm = 0; kmm < nk; ++kmm) {
                qA.push_back(sx + row(kmm, kj) * NV);
                qC.push_back(P->seg[SEG_Q] + ((i64)kj * nk + kmm) * S2 * NV);
            }
        B.perm({o, v, o, NV}, {ov * NV, NV, v * NV, 1}, qA, BUF_SCRATCH, {v * o * NV, o * NV, NV, 1}, qC, 1.0, 0.0);
    }
    const i64 blk = ov * ov;
    // ring: T1[ki][kj][j][a][i] = sum_km W1[ka][kj][km] R'[ki][km] + W2[ka][kj][km] Q'[ki][km]
    B.cur = "ip_ring_w1w2";
    {
        std::vector<i64> oA, oB, oC;
        for (int ki = 0; ki < nk; ++ki)
            for (int kj = 0; kj < nk; ++kj) {
                int ka = km.c(ki, K, kj);
                for (int kmm = 0; kmm < nk; ++kmm) {
                    oA.push_back(0 * h->wov_seg + (((i64)ka * nk + kj) * nk + kmm) * blk);
                    oB.push_back(P->seg[SEG_R] + ((i64)ki * nk + kmm) * S2 * NV);
                    oA.push_back(1 * h->wov_seg + (((i64)ka * nk + kj) * nk + kmm) * blk);
                    oB.push_back(P->seg[SEG_Q] + ((i64)ki * nk + kmm) * S2 * NV);
                }
                oC.push_back(P->seg[SEG_T1] + ((i64)ki * nk + kj) * S2 * NV);
            }
        B.gemm((int)ov, (int)(o * NV), (int)ov, 2 * nk, BUF_WOV3, ov, 1, oA, o * NV, 1, oB, BUF_SCRATCH, o * NV, 1, oC, 1.0,
               0.0);
        std::vector<i64> pA, pC;
        for (int ki = 0; ki < nk; ++ki)
            for (int kj = 0; kj < nk; ++kj) {
                pA.push_back(P->seg[SEG_T1] + ((i64)ki * nk + kj) * S2 * NV);
                pC.push_back(row(ki, kj) * NV);
            }
        // T1 [j][a][i] -> s2 [i][j][a]
        B.perm({o, v, o, NV}, {v * o * NV, o * NV, NV, 1}, pA, BUF_Y, {v * NV, NV, ov * NV, 1}, pC, 1.0, 1.0);
    }
    // ring: T3[ki][kj][i][a][j] = sum_km WN[ka][ki][km] Q'[kj][km]
    B.cur = "ip_ring_wn";
    {
        std::vector<i64> oA, oB, oC;
        for (int ki = 0; ki < nk; ++ki)
            for (int kj = 0; kj < nk; ++kj) {
                int ka = km.c(ki, K, kj);
                for (int kmm = 0; kmm < nk; ++kmm) {
                    oA.push_back(2 * h->wov_seg + (((i64)ka * nk + ki) * nk + kmm) * blk);
                    oB.push_back(P->seg[SEG_Q] + ((i64)kj * nk + kmm) * S2 * NV);
                }
                oC.push_back(P->seg[SEG_T3] + ((i64)ki * nk + kj) * S2 * NV);
            }
        B.gemm((int)ov, (int)(o * NV), (int)ov, nk, BUF_WOV3, ov, 1, oA, o * NV, 1, oB, BUF_SCRATCH, o * NV, 1, oC, 1.0, 0.0);
        std::vector<i64> pA, pC;
        for (int ki = 0; ki < nk; ++ki)
            for (int kj = 0; kj < nk; ++kj) {
                pA.push_back(P->seg[SEG_T3] + ((i64)ki * nk + kj) * S2 * NV);
                pC.push_back(row(ki, kj) * NV);
            }
        // T3 [i][a][j] -> s2 [i][j][a]
        B.perm({o, v, o, NV}, {v * o * NV, o * NV, NV, 1}, pA, BUF_Y, {ov * NV, NV, v * NV, 1}, pC, 1.0, 1.0);
    }
    // three-body: Xsm[e] = sum (2<mn|ef> - <mn|fe>) r2[km,kn][m,n,f];  s2 -= t2[ki,kj,K][i,j,e,a] Xsm[e]
    B.cur = "ip_threebody";
    {
        const i64 sm = P->seg[SEG_SMALL];
        B.gemm(v, nv, (int)(nk2 * S2), 1, BUF_UOOVV_IP, nk2 * S2, 1, {(i64)K * v * nk2 * S2}, NV, 1, {sx + o * NV},
               BUF_SCRATCH, NV, 1, {sm}, 1.0, 0.0);
        std::vector<i64> oA, oB, oC;
        for (int ki = 0; ki < nk; ++ki)
            for (int kj = 0; kj < nk; ++kj) {
                oA.push_back((((i64)ki * nk + kj) * nk + K) * S2 * v);
                oB.push_back(sm);
                oC.push_back(row(ki, kj) * NV);
            }
        B.gemm((int)S2, nv, v, 1, BUF_T2IP, v, 1, oA, NV, 1, oB, BUF_Y, NV, 1, oC, -1.0, 1.0);
    }
    P->host_off = B.off;
    return P;
}

// ---------------------------------------------------------------- Fov terms
// IP: y1[i] += sum_{km,m,e} f_me (2 x2[K,km][i,m,e] - x2[km,K][m,i,e])
// EA: y1[a] += sum_{km,m,e} f_me (2 x2[km,K][m,a,e] - x2[km,km][m,e,a])
// One block per output row p: thread (c0 = tid % cw, g = tid / cw) sums the terms t = g, g + G, ...
// of column c = c0 (+ cw, ...), the G partial sums are added in a fixed order (the few-row
// reduction has nk o v terms, too long for one thread per output).
template <typename T, typename R>
__global__ void fov_kernel(int sector, int K, int nk, int o, int v, int nv, int cw, const T *__restrict__ Fov,
                           const T *__restrict__ x, T *__restrict__ y) {
    __shared__ R red[2][256];
    const int p = blockIdx.x;
    const int c0 = (int)threadIdx.x % cw, g = (int)threadIdx.x / cw, G = (int)blockDim.x / cw;
    const int ov = o * v, nterm = nk * ov;
    for (int cb = 0; cb < nv; cb += cw) {
        const int c = cb + c0;
        R ax = 0, ay = 0;
        if (c < nv) {
            for (int t = g; t < nterm; t += G) {
                const int kmm = t / ov, m = (t / v) % o, e = t % v;
                const T f = Fov[((i64)kmm * o + m) * v + e];
                T u, w;
                if (sector == CCGF_SECTOR_IP) {
                    const i64 S2 = (i64)o * o * v;
                    u = x[(o + ((i64)K * nk + kmm) * S2 + (i64)(p * o + m) * v + e) * nv + c];
                    w = x[(o + ((i64)kmm * nk + K) * S2 + (i64)(m * o + p) * v + e) * nv + c];
                } else {
                    const i64 S2 = (i64)o * v * v;
                    u = x[(v + ((i64)kmm * nk + K) * S2 + (i64)(m * v + p) * v + e) * nv + c];
                    w = x[(v + ((i64)kmm * nk + kmm) * S2 + (i64)(m * v + e) * v + p) * nv + c];
                }
                const R zx = 2 * u.x - w.x, zy = 2 * u.y - w.y;
                ax += f.x * zx - f.y * zy;
                ay += f.x * zy + f.y * zx;
            }
        }
        red[0][threadIdx.x] = ax;
        red[1][threadIdx.x] = ay;
        __syncthreads();
        if (g == 0 && c < nv) {
            R sx = 0, sy = 0;
            for (int q = 0; q < G; ++q) {
                sx += red[0][q * cw + c0];
                sy += red[1][q * cw + c0];
            }
            T out = y[(i64)p * nv + c];
            out.x += sx;
            out.y += sy;
            y[(i64)p * nv + c] = out;
        }
        __syncthreads();
    }
}

// EA ladder, pair-symmetric form. Pair representatives reps[s][beta] = (ke * v + e) * v + f,
// first nmi[s] non-fixed pairs, then the fixed ones (ke = kf, e = f); kj = s - K.
template <typename T, typename R>
__global__ void ladder_gather_kernel(int K, int nk, int o, int v, int nv, const int *ksub, const int *reps, const int *npl,
                                     const int *nmi, int Pp, int Pm, const T *__restrict__ x, T *__restrict__ Rp,
                                     T *__restrict__ Rm) {
    const i64 S2 = (i64)o * v * v, total = (i64)nk * Pp * o * nv;
    for (i64 idx = (i64)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (i64)gridDim.x * blockDim.x) {
        const int vec = idx % nv, j = (idx / nv) % o;
        const int be = (int)((idx / ((i64)nv * o)) % Pp), s = (int)(idx / ((i64)nv * o * Pp));
        const int kj = ksub[s * nk + K];
        T rp, rm;
        rp.x = rp.y = rm.x = rm.y = 0;
        if (be < npl[s]) {
            const int rep = reps[(i64)s * Pp + be];
            const int ke = rep / (v * v), e = (rep / v) % v, f = rep % v, kf = ksub[s * nk + ke];
            const T r1 = x[(v + ((i64)kj * nk + ke) * S2 + ((i64)j * v + e) * v + f) * nv + vec];
            if (be < nmi[s]) {
                const T r2 = x[(v + ((i64)kj * nk + kf) * S2 + ((i64)j * v + f) * v + e) * nv + vec];
                rp.x = (R)0.5 * (r1.x + r2.x);
                rp.y = (R)0.5 * (r1.y + r2.y);
                rm.x = (R)0.5 * (r1.x - r2.x);
                rm.y = (R)0.5 * (r1.y - r2.y);
            } else {
                rp = r1;
            }
        }
        Rp[(((i64)s * Pp + be) * o + j) * nv + vec] = rp;
        if (be < Pm) Rm[(((i64)s * Pm + be) * o + j) * nv + vec] = rm;
    }
}
template <typename T, typename R>
__global__ void ladder_scatter_kernel(int K, int nk, int o, int v, int nv, const int *ksub, const int *reps, const int *npl,
                                      const int *nmi, int Pp, int Pm, const T *__restrict__ Sp, const T *__restrict__ Sm,
                                      T *__restrict__ y) {
    const i64 S2 = (i64)o * v * v, total = (i64)nk * Pp * o * nv;
    for (i64 idx = (i64)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (i64)gridDim.x * blockDim.x) {
        const int vec = idx % nv, j = (idx / nv) % o;
        const int al = (int)((idx / ((i64)nv * o)) % Pp), s = (int)(idx / ((i64)nv * o * Pp));
        if (al >= npl[s]) continue;
        const int kj = ksub[s * nk + K];
        const int rep = reps[(i64)s * Pp + al];
        const int ka = rep / (v * v), a = (rep / v) % v, b = rep % v, kb = ksub[s * nk + ka];
        const T sp = Sp[(((i64)s * Pp + al) * o + j) * nv + vec];
        T sm;
        sm.x = sm.y = 0;
        const bool nonfixed = al < nmi[s];
        if (nonfixed) sm = Sm[(((i64)s * Pm + al) * o + j) * nv + vec];
        T *y1 = y + (v + ((i64)kj * nk + ka) * S2 + ((i64)j * v + a) * v + b) * nv + vec;
        y1->x += sp.x + sm.x;
        y1->y += sp.y + sm.y;
        if (nonfixed) {
            T *y2 = y + (v + ((i64)kj * nk + kb) * S2 + ((i64)j * v + b) * v + a) * nv + vec;
            y2->x += sp.x - sm.x;
            y2->y += sp.y - sm.y;
        }
    }
}

template <typename R> using T_arena = typename cvec<R>::T *;

template <typename R>
__global__ void convert_kernel(const double2 *__restrict__ a, typename cvec<R>::T *__restrict__ b, i64 n) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
        typename cvec<R>::T t;
        t.x = (R)a[i].x;
        t.y = (R)a[i].y;
        b[i] = t;
    }
}
__global__ void widen_kernel(const float2 *__restrict__ a, double2 *__restrict__ b, i64 n) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
        b[i] = make_double2((double)a[i].x, (double)a[i].y);
}
inline unsigned gsz(i64 n) {
    i64 g = ceil_div(n, 256);
    return (unsigned)(g > 152 * 32 ? 152 * 32 : (g > 0 ? g : 1));
}

// GEMM kernel choices of a plan step: 0 = default (the bulk-fed tensor-core kernel when the A
// operand is TMA-addressable, else the register-fed one; SIMT tile by the launcher's model),
// k in 1..zgemm_tile_count() = SIMT kernel with the launcher's k-th tile, k + 1000 s = the same
// with K split over s CTAs (s >= 2, partial sums reduced by a second kernel), the few-row kernel
// (200), or one of the three tensor-core kernels (100-102)
enum { CHOICE_TC_TMA = 100, CHOICE_TC_REG = 101, CHOICE_TC_BULK = 102, CHOICE_TC_OZ = 103, CHOICE_SMALLM = 200, CHOICE_SPLIT = 1000 };

// one GEMM step with the given choice; returns the number of launches (0: choice not applicable)
template <typename R>
int run_gemm_step(ccgf_handle *h, const SigmaPlan *P, const SigmaStep &s, int choice, bool tensor_cores,
                  typename cvec<R>::T *scr, typename cvec<R>::T *yout, cudaStream_t st) {
    typedef typename cvec<R>::T T;
    const bool f64 = sizeof(R) == 8;
    const i64 *offs = P->offsets.p;
    T *C = s.c_buf == BUF_Y ? yout : scr;
    GemmDesc d = s.g;
    d.wait_ns = h->wait_ns;
    d.offA = offs + s.offA_pos;
    d.offB = offs + s.offB_pos;
    d.offC = offs + s.offC_pos;
    const T *A = f64 ? (const T *)h->W[s.a_buf].p : (const T *)h->Wf[s.a_buf].p;
    if constexpr (sizeof(R) == 4) {
        if (!A) {
            // no FP32 copy of this block (device memory): FP32 / TF32 arithmetic on the FP64 block
            if (tensor_cores && tc_zgemm_supported(d)) return launch_tc_zgemm_a64(d, h->W[s.a_buf].p, scr, C, h->tc_err.p, st);
            return launch_tgemm_a64(tgemm_of(d), h->W[s.a_buf].p, scr, C, st, scr + P->seg[SEG_SPLITK],
                                    P->seg[SEG_END] - P->seg[SEG_SPLITK]);
        }
    }
    if constexpr (sizeof(R) == 8) {
        // CCGF_FP64_TC: the FP64-accurate sliced tensor-core GEMM where the step allows it (the default)
        if (tensor_cores && (choice == 0 || choice == CHOICE_TC_OZ)) {
            int n = 0;
            if (s.rowA_pos >= 0)
                n = launch_tc_zgemm_oz(h, s.a_buf, d, offs + s.rowA_pos, offs + s.bslot_pos, offs + s.bsrc_pos, s.nslots, scr, C,
                                       h->tc_err.p, st);
            if (n > 0 || choice == CHOICE_TC_OZ) return n;
        }
    }
    if (choice == CHOICE_SMALLM) return launch_zgemm_smallm<R>(d, A, scr, C, st);
    if constexpr (sizeof(R) == 4) {
        if (tensor_cores && tc_zgemm_supported(d) && (choice == 0 || (choice >= CHOICE_TC_TMA && choice < CHOICE_SMALLM))) {
            int n = 0;
            if ((choice == 0 || choice == CHOICE_TC_BULK) && s.rowA_pos >= 0)
                n = launch_tc_zgemm_bulk(h, s.a_buf, d, offs + s.rowA_pos, offs + s.bslot_pos, offs + s.bsrc_pos, s.nslots, scr, C,
                                         h->tc_err.p, st);
            if (n == 0 && choice == CHOICE_TC_TMA && s.rowA_pos >= 0)
                n = launch_tc_zgemm_tma(h, s.a_buf, d, offs + s.rowA_pos, scr, C, h->tc_err.p, st);
            if (n == 0 && (choice == 0 || choice == CHOICE_TC_REG)) n = launch_tc_zgemm(d, A, scr, C, h->tc_err.p, st);
            return n;
        }
    }
    if (choice >= CHOICE_TC_TMA && choice < CHOICE_SPLIT) return 0;
    d.tile = choice % CHOICE_SPLIT;
    d.ksplit = choice / CHOICE_SPLIT;
    if (d.ksplit > 1) {
        // wave-filling split: partial sums in the handle's split workspace (sized by the autotuner;
        // the launcher runs unsplit if it is too small)
        if (f64) return launch_zgemm<R>(d, A, scr, C, st, (T *)h->splitw64.p, h->splitw64.n);
        return launch_zgemm<R>(d, A, scr, C, st, (T *)h->splitw32.p, h->splitw32.n);
    }
    return launch_zgemm<R>(d, A, scr, C, st, scr + P->seg[SEG_SPLITK], P->seg[SEG_END] - P->seg[SEG_SPLITK]);
}

// Measured kernel choice per GEMM step (an autotuner): every candidate (the SIMT tiles, the few-row
// kernel where it applies and, for
// CCGF_TF32X3, the two tensor-core kernels) runs once to warm up and twice timed with CUDA
// events on the real operands; the fastest is kept in the step and in a process-wide table keyed
// by the GEMM's shape, strides and precision, so later plans and handles reuse it without timing.
// Runs before the plan's first execution, when the scratch arena and the output hold no live data
// (every plan step writes its outputs before it reads them). CCGF_AUTOTUNE=0 keeps the defaults.
struct TuneKey {
    int pi, a_buf, M, N, K, nred, batch, tma;
    i64 rsA, csA, rsB, csB, rsC, csC;
    bool beta;
    bool operator<(const TuneKey &o) const {
        return std::tie(pi, a_buf, M, N, K, nred, batch, tma, rsA, csA, rsB, csB, rsC, csC, beta) <
               std::tie(o.pi, o.a_buf, o.M, o.N, o.K, o.nred, o.batch, o.tma, o.rsA, o.csA, o.rsB, o.csB, o.rsC, o.csC, o.beta);
    }
};
std::map<TuneKey, int> g_tuned;
std::mutex g_tuned_mu;

std::atomic<int> g_autotune{-1};   // -1: not read yet, then 0 / 1
bool autotune_enabled() {
    int v = g_autotune.load();
    if (v < 0) {
        const char *e = std::getenv("CCGF_AUTOTUNE");
        int want = (e && e[0] == '0') ? 0 : 1;
        g_autotune.compare_exchange_strong(v, want);
        v = g_autotune.load();
    }
    return v != 0;
}

// grows the handle's split-K workspace of this precision to hold a `choice` split of GEMM g
template <typename R> ccgf_status ensure_split_ws(ccgf_handle *h, const GemmDesc &g, int choice, cudaStream_t st) {
    if (choice < CHOICE_SPLIT) return CCGF_OK;
    GemmDesc d = g;
    d.tile = choice % CHOICE_SPLIT;
    d.ksplit = choice / CHOICE_SPLIT;
    const i64 need = zgemm_workspace_elems(d);
    const i64 cap = sizeof(R) == 8 ? h->splitw64.n : h->splitw32.n;
    if (need <= cap) return CCGF_OK;
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    if (sizeof(R) == 8) {
        dfree(h->splitw64);
        CCGF_TRY(dalloc(h->splitw64, need));
    } else {
        dfree(h->splitw32);
        CCGF_TRY(dalloc(h->splitw32, need));
    }
    return CCGF_OK;
}

template <typename R>
ccgf_status autotune_plan(ccgf_handle *h, SigmaPlan *P, int pi, bool tensor_cores, typename cvec<R>::T *scr,
                          typename cvec<R>::T *yout, cudaStream_t st) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = on_scope_exit([&] {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    });
    for (SigmaStep &s : P->steps) {
        if (s.kind != STEP_GEMM) continue;
        if (sizeof(R) == 4 && !h->Wf[s.a_buf].p) continue;   // converted on load: one kernel per precision
        if (s.choice[pi] != 0) {
            CCGF_TRY(ensure_split_ws<R>(h, s.g, s.choice[pi], st));
            continue;
        }
        const GemmDesc &g = s.g;
        TuneKey key{pi, s.a_buf, g.M, g.N, g.K, g.nred, g.batch, s.rowA_pos >= 0 ? 1 : 0,
                    g.rsA, g.csA, g.rsB, g.csB, g.rsC, g.csC, g.beta.x != 0.0 || g.beta.y != 0.0};
        {
            std::lock_guard<std::mutex> lk(g_tuned_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) s.choice[pi] = it->second;
        }
        if (s.choice[pi] != 0) {
            CCGF_TRY(ensure_split_ws<R>(h, s.g, s.choice[pi], st));
            continue;
        }
        if (!e0) {
            CCGF_CUDA_TRY(cudaEventCreate(&e0));
            CCGF_CUDA_TRY(cudaEventCreate(&e1));
        }
        // candidates, most promising first (the tensor-core kernels, then the launcher's own SIMT pick);
        // a contraction whose runs are long is tuned only until 1.5 s of timing has been spent
        std::vector<int> cand;
        const bool tc_ok = sizeof(R) == 4 && tensor_cores && tc_zgemm_supported(g);
        if (sizeof(R) == 8 && tensor_cores && s.rowA_pos >= 0 && tc_zgemm_oz_supported(g)) cand.push_back(CHOICE_TC_OZ);
        if (tc_ok) {
            if (s.rowA_pos >= 0) {
                cand.push_back(CHOICE_TC_BULK);
                cand.push_back(CHOICE_TC_TMA);
            }
            cand.push_back(CHOICE_TC_REG);
        }
        {
            GemmDesc gm = g;
            gm.tile = 0;
            gm.ksplit = 0;
            const int model = zgemm_model_tile(gm);
            if (model > 0) cand.push_back(model);
            for (int t = 1; t <= zgemm_tile_count(); ++t) {
                if (t != model) cand.push_back(t);
                const int ks = zgemm_wave_split(g, t);
                if (ks > 1) cand.push_back(t + CHOICE_SPLIT * ks);
            }
        }
        if (zgemm_smallm_supported(g)) cand.push_back(CHOICE_SMALLM);
        int best = 0;
        float best_ms = 1e30f, spent = 0.f;
        for (int c : cand) {
            if (spent > 1500.f && best != 0) break;
            CCGF_TRY(ensure_split_ws<R>(h, s.g, c, st));
            CCGF_CUDA_TRY(cudaEventRecord(e0, st));
            int n = run_gemm_step<R>(h, P, s, c, tensor_cores, scr, yout, st);
            CCGF_CUDA_TRY(cudaEventRecord(e1, st));
            if (n == 0) continue;
            h->launches += n;
            CCGF_CUDA_TRY(cudaEventSynchronize(e1));
            float first = 0.f;
            CCGF_CUDA_TRY(cudaEventElapsedTime(&first, e0, e1));
            spent += first;
            float ms = 1e30f;
            const int reps = first > 20.f ? 1 : 2;
            for (int rep = 0; rep < reps; ++rep) {
                CCGF_CUDA_TRY(cudaEventRecord(e0, st));
                h->launches += run_gemm_step<R>(h, P, s, c, tensor_cores, scr, yout, st);
                CCGF_CUDA_TRY(cudaEventRecord(e1, st));
                CCGF_CUDA_TRY(cudaEventSynchronize(e1));
                float t = 0.f;
                CCGF_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
                spent += t;
                ms = t < ms ? t : ms;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        s.choice[pi] = best;
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        g_tuned[key] = best;
    }
    return CCGF_OK;
}

template <typename R>
void run_plan(ccgf_handle *h, SigmaPlan *P, const double2 *x, double2 *y, cudaStream_t st, T_arena<R> arena = nullptr,
              bool tensor_cores = false) {
    typedef typename cvec<R>::T T;
    const bool f64 = sizeof(R) == 8;
    const int pi = f64 ? (tensor_cores ? 3 : 0) : (tensor_cores ? 2 : 1);
    T *scr = arena ? arena : (f64 ? (T *)h->scratch.p : (T *)h->scratch_f.p);
    const i64 D = P->sector == CCGF_SECTOR_IP ? h->dim_ip : h->dim_ea;
    const i64 n = D * P->nv;
    T *yout = f64 ? (T *)y : (T *)h->yf.p;
    // input -> scratch segment X (copy or narrowing conversion)
    convert_kernel<R><<<gsz(n), 256, 0, st>>>(x, scr + P->seg[SEG_X], n);
    h->launches++;
    const i64 *offs = P->offsets.p;
    int si = 0;
    for (const SigmaStep &s : P->steps) {
        if (h->prof_events && si < h->prof_max) cudaEventRecord(h->prof_events[si], st);
        ++si;
        T *C = s.c_buf == BUF_Y ? yout : scr;
        if (s.kind == STEP_GEMM) {
            int n = run_gemm_step<R>(h, P, s, s.choice[pi], tensor_cores, scr, yout, st);
            // the measured choice may need operand copies released since (release_caches): default kernel
            if (n == 0 && s.choice[pi] != 0) n = run_gemm_step<R>(h, P, s, 0, tensor_cores, scr, yout, st);
            h->launches += n;
        } else if (s.kind == STEP_TGEMM) {
            auto ptr = [&](int b) -> T * {
                if (b == BUF_Y) return yout;
                if (b == BUF_SCRATCH) return scr;
                return f64 ? (T *)h->W[b].p : (T *)h->Wf[b].p;
            };
            TGemm d = s.tg;
            d.offA = offs + s.offA_pos;
            d.offB = offs + s.offB_pos;
            d.offC = offs + s.offC_pos;
            h->launches += launch_tgemm<R>(d, ptr(s.a_buf), ptr(s.b_buf), ptr(s.c_buf), st, scr + P->seg[SEG_SPLITK],
                                           P->seg[SEG_END] - P->seg[SEG_SPLITK]);
        } else if (s.kind == STEP_PERM) {
            PermDesc d = s.p;
            d.offA = offs + s.offA_pos;
            d.offC = offs + s.offC_pos;
            h->launches += launch_zpermute<R>(d, scr, C, st);
        } else if (s.kind == STEP_LADDER_GATHER || s.kind == STEP_LADDER_SCATTER) {
            const i64 total = (i64)h->nk * h->lad_Pp * h->o * P->nv;
            if (s.kind == STEP_LADDER_GATHER)
                ladder_gather_kernel<T, R><<<gsz(total), 256, 0, st>>>(P->K, h->nk, h->o, h->v, P->nv, h->ksub_d.p, h->lad_reps.p,
                                                                     h->lad_npl.p, h->lad_nmi.p, h->lad_Pp, h->lad_Pm,
                                                                     scr + P->seg[SEG_X], scr + s.lad_rp, scr + s.lad_rm);
            else
                ladder_scatter_kernel<T, R><<<gsz(total), 256, 0, st>>>(P->K, h->nk, h->o, h->v, P->nv, h->ksub_d.p, h->lad_reps.p,
                                                                      h->lad_npl.p, h->lad_nmi.p, h->lad_Pp, h->lad_Pm,
                                                                      scr + s.lad_rp, scr + s.lad_rm, yout);
            h->launches++;
        } else {
            const int sector = s.kind == STEP_FOV_IP ? CCGF_SECTOR_IP : CCGF_SECTOR_EA;
            const int nrow = sector == CCGF_SECTOR_IP ? h->o : h->v;
            const T *F = f64 ? (const T *)h->W[BUF_FOV].p : (const T *)h->Wf[BUF_FOV].p;
            fov_kernel<T, R><<<(unsigned)nrow, (unsigned)((256 / std::min(P->nv, 256)) * std::min(P->nv, 256)), 0, st>>>(
                sector, P->K, h->nk, h->o, h->v, P->nv, std::min(P->nv, 256), F, scr + P->seg[SEG_X], yout);
            h->launches++;
        }
    }
    if (h->prof_events && si < h->prof_max) cudaEventRecord(h->prof_events[si], st);
    h->prof_count = si + 1;
    if (!f64) {
        widen_kernel<<<gsz(n), 256, 0, st>>>(h->yf.p, y, n);
        h->launches++;
    }
}

// Host-side proof that every access of every launch of a plan stays inside its buffer:
// for each batch entry the largest address is offset + sum (extent - 1) * |stride| (all strides
// are non-negative here), compared with the buffer length in complex elements.
bool check_plan(const ccgf_handle *h, const SigmaPlan *P, const std::vector<i64> &off, std::string &why) {
    const i64 D = P->sector == CCGF_SECTOR_IP ? h->dim_ip : h->dim_ea;
    const i64 ylen = D * P->nv, slen = P->scratch_elems;
    int si = 0;
    for (const SigmaStep &s : P->steps) {
        ++si;
        if (s.kind == STEP_GEMM) {
            const GemmDesc &g = s.g;
            const i64 alen = h->W[s.a_buf].n, clen = s.c_buf == BUF_Y ? ylen : slen;
            const i64 spanA = (i64)(g.M - 1) * g.rsA + (i64)(g.K - 1) * g.csA;
            const i64 spanB = (i64)(g.K - 1) * g.rsB + (i64)(g.N - 1) * g.csB;
            const i64 spanC = (i64)(g.M - 1) * g.rsC + (i64)(g.N - 1) * g.csC;
            for (int b = 0; b < g.batch; ++b) {
                for (int r = 0; r < g.nred; ++r) {
                    i64 oa = off[s.offA_pos + (i64)b * g.nred + r], ob = off[s.offB_pos + (i64)b * g.nred + r];
                    if (oa < 0 || oa + spanA >= alen) { why = "gemm A out of range at step " + std::to_string(si); return false; }
                    if (ob < 0 || ob + spanB >= slen) { why = "gemm B out of range at step " + std::to_string(si); return false; }
                }
                i64 oc = off[s.offC_pos + b];
                if (oc < 0 || oc + spanC >= clen) { why = "gemm C out of range at step " + std::to_string(si); return false; }
            }
        } else if (s.kind == STEP_TGEMM) {
            const TGemm &g = s.tg;
            auto len = [&](int b) -> i64 { return b == BUF_Y ? ylen : (b == BUF_SCRATCH ? slen : h->W[b].n); };
            const i64 la = len(s.a_buf), lb = len(s.b_buf), lc = len(s.c_buf);
            const i64 spanA = imap_span(g.am, g.M) + imap_span(g.ak, g.K), spanB = imap_span(g.bk, g.K) + imap_span(g.bn, g.N),
                      spanC = imap_span(g.cm, g.M) + imap_span(g.cn, g.N);
            if (s.b_buf != BUF_SCRATCH && s.b_buf < BUF_FOO) { why = "tensor GEMM B operand at step " + std::to_string(si); return false; }
            for (int b = 0; b < g.batch; ++b) {
                for (int r = 0; r < g.nred; ++r) {
                    i64 oa = off[s.offA_pos + (i64)b * g.nred + r], ob = off[s.offB_pos + (i64)b * g.nred + r];
                    if (oa < 0 || oa + spanA >= la) { why = "tensor GEMM A out of range at step " + std::to_string(si); return false; }
                    if (ob < 0 || ob + spanB >= lb) { why = "tensor GEMM B out of range at step " + std::to_string(si); return false; }
                }
                i64 oc = off[s.offC_pos + b];
                if (oc < 0 || oc + spanC >= lc) { why = "tensor GEMM C out of range at step " + std::to_string(si); return false; }
            }
        } else if (s.kind == STEP_LADDER_GATHER || s.kind == STEP_LADDER_SCATTER) {
            // segments: R+/S+ need nk Pp nocc nv, R-/S- need nk Pm nocc nv elements; x2 / y2 indices
            // come from representatives of the pair space, all inside [nvir, dim_ea) rows
            const i64 need_p = (i64)h->nk * h->lad_Pp * h->o * P->nv, need_m = (i64)h->nk * h->lad_Pm * h->o * P->nv;
            auto seg_len = [&](i64 off) -> i64 {
                for (int g = 0; g < SEG_END; ++g)
                    if (P->seg[g] == off) return P->seg[g + 1] - off;
                return -1;
            };
            if (P->sector != CCGF_SECTOR_EA || seg_len(s.lad_rp) < need_p || seg_len(s.lad_rm) < need_m) {
                why = "ladder segment too small at step " + std::to_string(si);
                return false;
            }
        } else if (s.kind == STEP_PERM) {
            const PermDesc &p = s.p;
            i64 spanA = 0, spanC = 0;
            for (int d = 0; d < p.nd; ++d) {
                spanA += (p.dims[d] - 1) * p.sA[d];
                spanC += (p.dims[d] - 1) * p.sC[d];
            }
            const i64 clen = s.c_buf == BUF_Y ? ylen : slen;
            for (int b = 0; b < p.batch; ++b) {
                i64 oa = off[s.offA_pos + b], oc = off[s.offC_pos + b];
                if (oa < 0 || oa + spanA >= slen) { why = "permute source out of range at step " + std::to_string(si); return false; }
                if (oc < 0 || oc + spanC >= clen) { why = "permute destination out of range at step " + std::to_string(si); return false; }
            }
        }
    }
    return true;
}

}  // namespace


static const SigmaPlan *plan_of(const ccgf_handle *h, int sector, int K) {
    if (h->plans.empty() || K < 0 || K >= h->nk || (sector != 1 && sector != 2)) return nullptr;
    return h->plans[(sector - 1) * h->nk + K];
}
int plan_step_count(const ccgf_handle *h, int sector, int K) {
    const SigmaPlan *P = plan_of(h, sector, K);
    return P ? (int)P->steps.size() : 0;
}
double plan_step_flops(const ccgf_handle *h, int sector, int K, int step) {
    const SigmaPlan *P = plan_of(h, sector, K);
    if (!P || step < 0 || step >= (int)P->steps.size()) return 0.0;
    const SigmaStep &s = P->steps[step];
    if (s.kind == STEP_GEMM) return 8.0 * s.g.M * (double)s.g.N * s.g.K * s.g.nred * s.g.batch;
    if (s.kind == STEP_TGEMM) return 8.0 * s.tg.M * (double)s.tg.N * s.tg.K * s.tg.nred * s.tg.batch;
    if (s.kind == STEP_FOV_IP || s.kind == STEP_FOV_EA) {
        double rows = s.kind == STEP_FOV_IP ? h->o : h->v;
        return 8.0 * rows * P->nv * h->nk * h->o * h->v;
    }
    return 0.0;
}
const char *plan_step_name(const ccgf_handle *h, int sector, int K, int step) {
    const SigmaPlan *P = plan_of(h, sector, K);
    if (!P || step < 0 || step >= (int)P->steps.size()) return "";
    return P->steps[step].name;
}

void set_autotune(bool on) { g_autotune.store(on ? 1 : 0); }
int plan_step_choice(const ccgf_handle *h, int sector, int K, int step, int pi) {
    const SigmaPlan *P = plan_of(h, sector, K);
    if (!P || step < 0 || step >= (int)P->steps.size() || pi < 0 || pi > 3) return -1;
    const SigmaStep &s = P->steps[step];
    if (s.kind == STEP_TGEMM) return 400;
    if (s.kind != STEP_GEMM) return -1;
    if ((pi == 1 || pi == 2) && !h->Wf[s.a_buf].p) {
        // FP64-stored block (no FP32 copy): register-fed tensor cores or the tensor GEMM, rounding on load
        GemmDesc d = s.g;
        return (pi == 2 && tc_zgemm_supported(d)) ? 300 : 301;
    }
    return s.choice[pi];
}

// Drops what the handle keeps only for speed and rebuilds on demand: the FP32 copies of the
// intermediates (ensure_fp32), their TF32 hi / lo splits (tc_prepare), the sliced planes of the
// FP64-accurate tensor-core path, the sigma scratch arenas and the split-K workspaces.
// Synchronises the device (cudaFree).
void release_caches(ccgf_handle *h) {
    tc_free(h);
    oz_free(h);
    vcache_free(h);
    for (int b = 0; b < NBUF; ++b) dfree(h->Wf[b]);
    h->fp32_done = false;
    dfree(h->scratch);
    dfree(h->scratch_f);
    dfree(h->yf);
    dfree(h->splitw64);
    dfree(h->splitw32);
    // not the ABI transposes: a sigma call that releases the caches is reading and writing them
}

void free_plans(ccgf_handle *h) {
    for (SigmaPlan *p : h->plans)
        if (p) {
            dfree(p->offsets);
            delete p;
        }
    h->plans.assign(h->plans.size(), nullptr);
}

// FP32 copies of the intermediates for the low-precision sigma, smallest first. The operands of the
// tensor GEMMs and every block under 1 GB always get one; a larger block gets one only while at least
// `reserve` bytes of device memory stay free afterwards, else its GEMMs read the FP64 block and round
// it as it is loaded (tgemm_a64 / the register-fed tensor-core kernel), with the same result.
ccgf_status ensure_fp32(ccgf_handle *h, cudaStream_t st, size_t reserve) {
    if (h->fp32_done) return CCGF_OK;
    std::vector<int> order;
    for (int b = BUF_FOO; b < NBUF; ++b)
        if (h->W[b].p && !h->Wf[b].p) order.push_back(b);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return h->W[a].n < h->W[b].n; });
    for (int b : order) {
        const size_t bytes = (size_t)h->W[b].n * sizeof(float2);
        const bool needed = b == BUF_LD || b == BUF_OVOV || b == BUF_T2 || bytes < ((size_t)1 << 30);
        if (!needed) {
            size_t fr = 0, tot = 0;
            CCGF_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
            if (fr < bytes + reserve) continue;
        }
        CCGF_TRY(dalloc(h->Wf[b], h->W[b].n));
        convert_kernel<float><<<gsz(h->W[b].n), 256, 0, st>>>(h->W[b].p, h->Wf[b].p, h->W[b].n);
        h->launches++;
    }
    h->fp32_done = true;
    CCGF_CUDA_TRY(cudaGetLastError());
    return CCGF_OK;
}

ccgf_status sigma_apply(ccgf_handle *h, int sector, int K, int nv, const double2 *x, double2 *y, ccgf_precision prec,
                        cudaStream_t st) {
    if (nv != h->plan_nv) {
        // plans and scratch are sized for nv columns; rebuild on change
        CCGF_CUDA_TRY(cudaStreamSynchronize(st));
        free_plans(h);
        h->plan_nv = nv;
    }
    if (h->plans.empty()) h->plans.assign(2 * h->nk, nullptr);
    SigmaPlan *&P = h->plans[(sector - 1) * h->nk + K];
    if (!P) {
        SigmaPlan *np = sector == CCGF_SECTOR_IP ? build_plan_ip(h, K, nv) : build_plan_ea(h, K, nv);
        std::string why;
        if (!check_plan(h, np, np->host_off, why)) {
            delete np;
            set_last_error("internal sigma plan failed its bound check: " + why);
            return CCGF_ERR_INVALID_ARG;
        }
        ccgf_status s = dalloc(np->offsets, (i64)np->host_off.size());
        if (s != CCGF_OK) { delete np; return s; }
        CCGF_CUDA_TRY(cudaMemcpy(np->offsets.p, np->host_off.data(), sizeof(i64) * np->host_off.size(), cudaMemcpyHostToDevice));
        P = np;
    }
    const i64 D = sector == CCGF_SECTOR_IP ? h->dim_ip : h->dim_ea;
    if (prec == CCGF_FP64 || prec == CCGF_FP64_TC) {
        const bool tc = prec == CCGF_FP64_TC;
        if (tc && !h->tc_err.p) {
            CCGF_TRY(dalloc(h->tc_err, 1));
            CCGF_CUDA_TRY(cudaMemset(h->tc_err.p, 0, sizeof(int)));
        }
        if (h->scratch.n < P->scratch_elems) {
            CCGF_CUDA_TRY(cudaStreamSynchronize(st));
            dfree(h->scratch);
            if (dalloc(h->scratch, P->scratch_elems) != CCGF_OK) {
                // low-precision copies made by earlier calls give way to the FP64 scratch
                release_caches(h);
                CCGF_TRY(dalloc(h->scratch, P->scratch_elems));
            }
        }
        if (autotune_enabled()) CCGF_TRY(autotune_plan<double>(h, P, tc ? 3 : 0, tc, (double2 *)h->scratch.p, y, st));
        run_plan<double>(h, P, x, y, st, nullptr, tc);
    } else {
        if (h->scratch_f.n < P->scratch_elems || h->yf.n < D * nv) {
            CCGF_CUDA_TRY(cudaStreamSynchronize(st));
            const i64 dmax = h->dim_ip > h->dim_ea ? h->dim_ip : h->dim_ea;
            auto grow = [&]() -> ccgf_status {
                if (h->scratch_f.n < P->scratch_elems) {
                    dfree(h->scratch_f);
                    CCGF_TRY(dalloc(h->scratch_f, P->scratch_elems));
                }
                if (h->yf.n < dmax * nv) {
                    dfree(h->yf);
                    CCGF_TRY(dalloc(h->yf, dmax * nv));
                }
                return CCGF_OK;
            };
            if (grow() != CCGF_OK) {
                // copies made by earlier calls give way (they are made again below, as memory allows)
                release_caches(h);
                CCGF_TRY(grow());
            }
        }
        CCGF_TRY(ensure_fp32(h, st, (size_t)2 << 30));
        const bool tc = prec == CCGF_TF32X3;
        if (tc && !h->tc_err.p) {
            CCGF_TRY(dalloc(h->tc_err, 1));
            CCGF_CUDA_TRY(cudaMemset(h->tc_err.p, 0, sizeof(int)));
        }
        if (tc) CCGF_TRY(tc_prepare(h, st, (size_t)2 << 30));
        if (autotune_enabled()) CCGF_TRY(autotune_plan<float>(h, P, tc ? 2 : 1, tc, h->scratch_f.p, h->yf.p, st));
        run_plan<float>(h, P, x, y, st, nullptr, tc);
    }
    CCGF_CUDA_TRY(cudaGetLastError());
    return CCGF_OK;
}


// W_vvvo[K] of the stored form: the EA r1 -> r2 plan applied to the v unit vectors of r1, its r2
// part kept as rows (kj, ka, j, a, b) x columns e, for every K
ccgf_status build_wvvvo_by_plan(ccgf_handle *h, cudaStream_t st) {
    const int nk = h->nk, v = h->v;
    const i64 D = h->dim_ea, R2 = D - v;
    CCGF_TRY(dalloc(h->W[BUF_WVVVO], (i64)nk * R2 * v));
    DBuf<double2> x, y, arena;
    CCGF_TRY(dalloc(x, D * v));
    CCGF_TRY(dalloc(y, D * v));
    CCGF_CUDA_TRY(cudaMemsetAsync(x.p, 0, sizeof(double2) * D * v, st));
    {
        std::vector<double2> eye((size_t)v * v, make_double2(0.0, 0.0));
        for (int e = 0; e < v; ++e) eye[(size_t)e * v + e] = make_double2(1.0, 0.0);
        CCGF_CUDA_TRY(cudaMemcpyAsync(x.p, eye.data(), sizeof(double2) * eye.size(), cudaMemcpyHostToDevice, st));
    }
    for (int K = 0; K < nk; ++K) {
        std::unique_ptr<SigmaPlan> P(build_plan_ea(h, K, v, true));
        std::string why;
        if (!check_plan(h, P.get(), P->host_off, why)) {
            set_last_error("internal W_vvvo plan failed its bound check: " + why);
            return CCGF_ERR_INVALID_ARG;
        }
        if (arena.n < P->scratch_elems) CCGF_TRY(dalloc(arena, P->scratch_elems));
        CCGF_TRY(dalloc(P->offsets, (i64)P->host_off.size()));
        CCGF_CUDA_TRY(cudaMemcpyAsync(P->offsets.p, P->host_off.data(), sizeof(i64) * P->host_off.size(), cudaMemcpyHostToDevice, st));
        run_plan<double>(h, P.get(), x.p, y.p, st, arena.p);
        CCGF_CUDA_TRY(cudaMemcpyAsync(h->W[BUF_WVVVO].p + (i64)K * R2 * v, y.p + (i64)v * v, sizeof(double2) * R2 * v,
                                      cudaMemcpyDeviceToDevice, st));
        CCGF_CUDA_TRY(cudaStreamSynchronize(st));   // the plan's offset table and the arena are reused
    }
    CCGF_CUDA_TRY(cudaGetLastError());
    return CCGF_OK;
}

ccgf_status tc_error_check(ccgf_handle *h, cudaStream_t st) {
    if (!h->tc_err.p) return CCGF_OK;
    int flag = 0;
    CCGF_CUDA_TRY(cudaMemcpyAsync(&flag, h->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    if (flag) {
        CCGF_CUDA_TRY(cudaMemsetAsync(h->tc_err.p, 0, sizeof(int), st));
        set_last_error("a tensor-core GEMM wait exceeded its limit (ccgf_options::device_wait_timeout_ms); its output tile was not written");
        return CCGF_ERR_TIMEOUT;
    }
    return CCGF_OK;
}

// Sigma with caller-provided device workspace: the plan is built on the host only,
// its offset table is copied into `offsets` (capacity in entries) and every scratch
// segment lives in `arena` (capacity in complex elements). No device allocation.
ccgf_status sigma_apply_in_arena(ccgf_handle *h, int sector, int K, int nv, const double2 *x, double2 *y, double2 *arena,
                                 i64 arena_elems, i64 *offsets, i64 offsets_cap, cudaStream_t st) {
    SigmaPlan *P = sector == CCGF_SECTOR_IP ? build_plan_ip(h, K, nv) : build_plan_ea(h, K, nv);
    if (P->scratch_elems > arena_elems || (i64)P->host_off.size() > offsets_cap) {
        i64 need = P->scratch_elems, noff = (i64)P->host_off.size();
        delete P;
        set_last_error("workspace too small for this nvec: needs " + std::to_string(need) + " complex elements and " +
                       std::to_string(noff) + " offsets");
        return CCGF_ERR_INVALID_ARG;
    }
    std::string why;
    if (!check_plan(h, P, P->host_off, why)) {
        delete P;
        set_last_error("internal sigma plan failed its bound check: " + why);
        return CCGF_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaMemcpyAsync(offsets, P->host_off.data(), sizeof(i64) * P->host_off.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        delete P;
        set_last_error(std::string("offset table copy: ") + cudaGetErrorString(e));
        return CCGF_ERR_CUDA;
    }
    P->offsets.p = offsets;   // borrowed, not owned
    run_plan<double>(h, P, x, y, st, arena);
    P->offsets.p = nullptr;
    delete P;
    CCGF_CUDA_TRY(cudaGetLastError());
    return CCGF_OK;
}

// FP64 scratch of the sigma plans per right-hand-side column (the larger of the two sectors)
i64 sigma_scratch_per_column(const ccgf_handle *h) {
    i64 seg[SEG_END + 1];
    scratch_layout(h, 1, seg, h->direct);
    return seg[SEG_END];
}

i64 sigma_arena_elems(const ccgf_handle *h, int nv) {
    i64 seg[SEG_END + 1];
    scratch_layout(h, nv, seg, false);
    return seg[SEG_END];
}
