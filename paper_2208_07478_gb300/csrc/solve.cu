// Batched restarted GMRES for the shifted EOM systems of Eq. 6 and the G contraction of Eq. 7 / Eq. 9.
//
// For one sector and total momentum K, the right-hand sides are all orbitals p times a chunk of
// frequencies; column c = p * nw + w of the [D][nv] arrays. Per column the operator is
//   M_c = z_c + s A,  z_c = w_c - i eta, s = +1 (IP);   z_c = w_c + i eta, s = -1 (EA),
// right-preconditioned by the diagonal P_c = 1 / (z_c + s d) with d the one-body part of diag(A).
// The Krylov basis, the CGS2 orthogonalisation, the Hessenberg / Givens least squares and the
// solution are FP64; the inner sigma runs in the requested precision. With a low-precision inner
// sigma a cycle that reaches the target of the low-precision iteration is followed by the FP64 true
// residual b - M x (iterative refinement; only that residual decides convergence; once a check has
// failed, the low-precision iteration aims at a tenth of the target), a cycle cut by the restart
// length restarts from the low-precision residual. All loops are host-driven (one
// small device->host read per Arnoldi step): no device code waits on anything.
//
// On this part FP64 arithmetic (2 DFMA per SM and clock) rather than HBM bounds the vector steps:
// a complex multiply-add on 16 bytes costs 4 DFMA, so the per-element kernels avoid FP64 division
// (the preconditioner is a table made once per batch, normalisation multiplies by a reciprocal
// per column) and 64-bit integer division (a thread keeps its column for the whole loop).
#include "ccgf_internal.h"
#include <algorithm>
#include <cmath>
#include <vector>

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cdiv1(double2 z) {   // 1 / z
    double den = z.x * z.x + z.y * z.y;
    return make_double2(z.x / den, -z.y / den);
}

struct Shift {
    const double2 *z;   // [nv]
    double s;           // +1 IP, -1 EA
    const double *d;    // [D] diagonal estimate
};
__device__ __forceinline__ double2 precond(const Shift &S, i64 mu, int c) {
    double2 z = S.z[c];
    return cdiv1(make_double2(z.x + S.s * S.d[mu], z.y));
}

// Per-element kernels over [D][nv] arrays: a block of cw * ry threads; thread (c0 = tid % cw,
// y = tid / cw) takes columns c0, c0 + cw, ... of rows y, y + ry, ... of its block's row groups, so a
// block reads ry * nv contiguous elements per group and no thread divides by nv in its loop.
#define ROW_LOOP(D, nv, cw, ry)                                                                   \
    const int c0_ = (int)threadIdx.x % (cw), y_ = (int)threadIdx.x / (cw);                        \
    for (i64 mu = (i64)blockIdx.x * (ry) + y_; mu < (D); mu += (i64)gridDim.x * (ry))             \
        for (int c = c0_; c < (nv); c += (cw))

// diag estimate: IP r1 -Foo_ii, r2 Fvv_aa - Foo_ii - Foo_jj;  EA r1 Fvv_aa, r2 Fvv_aa + Fvv_bb - Foo_jj
__global__ void diag_kernel(int sector, int K, int nk, int o, int v, const int *kadd, const int *ksub, const double2 *Foo,
                            const double2 *Fvv, double *d, i64 D) {
    for (i64 mu = (i64)blockIdx.x * blockDim.x + threadIdx.x; mu < D; mu += (i64)gridDim.x * blockDim.x) {
        double r;
        if (sector == CCGF_SECTOR_IP) {
            if (mu < o) r = -Foo[((i64)K * o + mu) * o + mu].x;
            else {
                i64 e = mu - o;
                int a = e % v; e /= v;
                int j = e % o; e /= o;
                int i = e % o; e /= o;
                int kj = e % nk, ki = (int)(e / nk);
                int ka = kadd[ksub[ki * nk + K] * nk + kj];
                r = Fvv[((i64)ka * v + a) * v + a].x - Foo[((i64)ki * o + i) * o + i].x - Foo[((i64)kj * o + j) * o + j].x;
            }
        } else {
            if (mu < v) r = Fvv[((i64)K * v + mu) * v + mu].x;
            else {
                i64 e = mu - v;
                int b = e % v; e /= v;
                int a = e % v; e /= v;
                int j = e % o; e /= o;
                int ka = e % nk, kj = (int)(e / nk);
                int kb = kadd[ksub[K * nk + ka] * nk + kj];
                r = Fvv[((i64)ka * v + a) * v + a].x + Fvv[((i64)kb * v + b) * v + b].x - Foo[((i64)kj * o + j) * o + j].x;
            }
        }
        d[mu] = r;
    }
}

// B[mu][c] = b_p[mu] for column c = (p - p0) * nw + w (zero for the padding columns p >= pend)
__global__ void expand_kernel(const double2 *Bq, double2 *B, i64 D, int N, int pend, int p0, int nw, int nv) {
    for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t < D * nv; t += (i64)gridDim.x * blockDim.x) {
        i64 mu = t / nv;
        int c = t % nv;
        const int p = p0 + c / nw;
        B[t] = p < pend ? Bq[mu * N + p] : make_double2(0.0, 0.0);
    }
}

// out[c] += sum_mu |v[mu][c]|^2   (out zeroed by the caller)
__global__ void colnorm2_kernel(const double2 *__restrict__ v, double *out, i64 D, int nv, i64 rows_per_block) {
    const int c = blockIdx.x * 32 + threadIdx.x;
    const i64 r0 = (i64)blockIdx.y * rows_per_block;
    const i64 r1 = min(D, r0 + rows_per_block);
    double acc = 0;
    if (c < nv)
        for (i64 mu = r0 + threadIdx.y; mu < r1; mu += 8) {
            double2 x = v[mu * nv + c];
            acc += x.x * x.x + x.y * x.y;
        }
    __shared__ double red[8][33];
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && c < nv) {
        double s = 0;
        for (int k = 0; k < 8; ++k) s += red[k][threadIdx.x];
        atomicAdd(out + c, s);
    }
}

// h[c][i] += sum_mu conj(V_i[mu][c]) w[mu][c], i = 0..J-1 (h zeroed by the caller)
__global__ void cgs_dot_kernel(const double2 *__restrict__ V, i64 vstride, const double2 *__restrict__ w, double2 *h, int hld,
                               int J, i64 D, int nv, i64 rows_per_block) {
    const int c = blockIdx.x * 32 + threadIdx.x;
    const i64 r0 = (i64)blockIdx.y * rows_per_block;
    const i64 r1 = min(D, r0 + rows_per_block);
    __shared__ double2 red[8][8][33];
    for (int i0 = 0; i0 < J; i0 += 8) {
        double2 acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = make_double2(0, 0);
        if (c < nv)
            for (i64 mu = r0 + threadIdx.y; mu < r1; mu += 8) {
                double2 x = w[mu * nv + c];
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (i0 + k < J) {
                        double2 vv = V[(i64)(i0 + k) * vstride + mu * nv + c];
                        double2 p = cconjmul(vv, x);
                        acc[k].x += p.x;
                        acc[k].y += p.y;
                    }
            }
#pragma unroll
        for (int k = 0; k < 8; ++k) red[k][threadIdx.y][threadIdx.x] = acc[k];
        __syncthreads();
        if (threadIdx.y < 8 && c < nv) {
            int k = threadIdx.y;
            if (i0 + k < J) {
                double2 s = make_double2(0, 0);
                for (int t = 0; t < 8; ++t) {
                    s.x += red[k][t][threadIdx.x].x;
                    s.y += red[k][t][threadIdx.x].y;
                }
                atomicAdd(&h[(i64)c * hld + i0 + k].x, s.x);
                atomicAdd(&h[(i64)c * hld + i0 + k].y, s.y);
            }
        }
        __syncthreads();
    }
}

// Partial CGS dot products without atomics: a block of nv * ry threads (thread = column c, row lane y)
// walks rows [b * rpb, (b + 1) * rpb) of the [D][nv] arrays, so a warp reads contiguous memory with
// every lane busy whatever nv is; part[b][i][c] = sum over the block's rows of conj(V_i[mu][c]) w[mu][c].
// rows [r0, r1) of one CGS chunk of NK basis vectors: acc[k] += conj(V_{i0+k}[mu][c]) w[mu][c]. NK is a
// template argument so that exactly NK products run per element (a predicated product still
// occupies the FP64 pipe, which bounds these kernels on this part).
template <int NK>
__device__ __forceinline__ void dot_rows(const double2 *__restrict__ V, i64 vstride, const double2 *__restrict__ w, int i0, i64 r0,
                                         i64 r1, int y, int ry, int nv, int c, double2 (&acc)[8]) {
    for (i64 mu = r0 + y; mu < r1; mu += ry) {
        const i64 t = mu * nv + c;
        const double2 x = w[t];
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const double2 vv = V[(i64)(i0 + k) * vstride + t];
            acc[k].x += vv.x * x.x + vv.y * x.y;
            acc[k].y += vv.x * x.y - vv.y * x.x;
        }
    }
}

__global__ void __launch_bounds__(256) ortho_dot_kernel(const double2 *__restrict__ V, i64 vstride, const double2 *__restrict__ w,
                                                         double2 *__restrict__ part, int J, i64 D, int nv, int ry, i64 rpb) {
    extern __shared__ double2 red[];                    // [ry][8][nv]
    const int c = threadIdx.x % nv, y = threadIdx.x / nv;
    const i64 r0 = (i64)blockIdx.x * rpb, r1 = min(D, r0 + rpb);
    for (int i0 = 0; i0 < J; i0 += 8) {
        double2 acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = make_double2(0, 0);
        if (y < ry) {
            switch (min(8, J - i0)) {
            case 1: dot_rows<1>(V, vstride, w, i0, r0, r1, y, ry, nv, c, acc); break;
            case 2: dot_rows<2>(V, vstride, w, i0, r0, r1, y, ry, nv, c, acc); break;
            case 3: dot_rows<3>(V, vstride, w, i0, r0, r1, y, ry, nv, c, acc); break;
            case 4: dot_rows<4>(V, vstride, w, i0, r0, r1, y, ry, nv, c, acc); break;
            case 5: dot_rows<5>(V, vstride, w, i0, r0, r1, y, ry, nv, c, acc); break;
            case 6: dot_rows<6>(V, vstride, w, i0, r0, r1, y, ry, nv, c, acc); break;
            case 7: dot_rows<7>(V, vstride, w, i0, r0, r1, y, ry, nv, c, acc); break;
            default: dot_rows<8>(V, vstride, w, i0, r0, r1, y, ry, nv, c, acc); break;
            }
        }
        if (y < ry)
#pragma unroll
            for (int k = 0; k < 8; ++k) red[((i64)y * 8 + k) * nv + c] = acc[k];
        __syncthreads();
        for (int e = threadIdx.x; e < 8 * nv; e += blockDim.x) {
            const int k = e / nv, cc = e % nv;
            if (i0 + k < J) {
                double2 sacc = make_double2(0, 0);
                for (int yy = 0; yy < ry; ++yy) {
                    const double2 q = red[((i64)yy * 8 + k) * nv + cc];
                    sacc.x += q.x;
                    sacc.y += q.y;
                }
                part[((i64)blockIdx.x * J + i0 + k) * nv + cc] = sacc;
            }
        }
        __syncthreads();
    }
}
// h[c][i] (+)= sum_b part[b][i][c]: one warp per (i, c), lanes over the blocks' partial sums (fixed
// order, so the result does not depend on timing), then a shuffle reduction
__global__ void ortho_sum_kernel(const double2 *__restrict__ part, int nblk, double2 *h, int hld, int J, int nv, int accumulate) {
    const int lane = threadIdx.x & 31;
    for (int e = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); e < J * nv; e += (int)((gridDim.x * blockDim.x) >> 5)) {
        const int i = e / nv, c = e % nv;
        double2 sacc = make_double2(0, 0);
        for (int b = lane; b < nblk; b += 32) {
            const double2 q = part[((i64)b * J + i) * nv + c];
            sacc.x += q.x;
            sacc.y += q.y;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sacc.x += __shfl_xor_sync(0xffffffffu, sacc.x, off);
            sacc.y += __shfl_xor_sync(0xffffffffu, sacc.y, off);
        }
        if (lane == 0) {
            double2 *o = h + (i64)c * hld + i;
            if (accumulate) {
                o->x += sacc.x;
                o->y += sacc.y;
            } else {
                *o = sacc;
            }
        }
    }
}

// w[mu][c] -= sum_{i<J} h[c][i] V_i[mu][c]
__global__ void cgs_axpy_kernel(const double2 *__restrict__ V, i64 vstride, double2 *w, const double2 *__restrict__ h, int hld,
                                int J, i64 D, int nv, int cw, int ry) {
    ROW_LOOP(D, nv, cw, ry) {
        const i64 t = mu * nv + c;
        const double2 *hc = h + (i64)c * hld;
        double2 acc = w[t];
        for (int i = 0; i < J; ++i) {
            const double2 p = cmul(hc[i], V[(i64)i * vstride + t]);
            acc.x -= p.x;
            acc.y -= p.y;
        }
        w[t] = acc;
    }
}

// preconditioner table P[mu][c] = 1 / (z_c + s d_mu), made once per batch
__global__ void ptab_kernel(Shift S, double2 *P, i64 D, int nv, int cw, int ry) {
    ROW_LOOP(D, nv, cw, ry) P[mu * nv + c] = precond(S, mu, c);
}
// U = P . V   (preconditioned direction)
__global__ void precond_kernel(const double2 *__restrict__ P, const double2 *__restrict__ V, double2 *U, i64 D, int nv, int cw,
                               int ry) {
    ROW_LOOP(D, nv, cw, ry) {
        const i64 t = mu * nv + c;
        U[t] = cmul(P[t], V[t]);
    }
}
// w = z U + s sigma(U)
__global__ void shift_kernel(Shift S, const double2 *__restrict__ U, const double2 *__restrict__ AU, double2 *w, i64 D, int nv,
                             int cw, int ry) {
    ROW_LOOP(D, nv, cw, ry) {
        const i64 t = mu * nv + c;
        const double2 zu = cmul(S.z[c], U[t]);
        const double2 a = AU[t];
        w[t] = make_double2(zu.x + S.s * a.x, zu.y + S.s * a.y);
    }
}
// r = b - (z x + s sigma(x))
__global__ void residual_kernel(Shift S, const double2 *__restrict__ b, const double2 *__restrict__ x,
                                const double2 *__restrict__ Ax, double2 *r, i64 D, int nv, int cw, int ry) {
    ROW_LOOP(D, nv, cw, ry) {
        const i64 t = mu * nv + c;
        const double2 zx = cmul(S.z[c], x[t]);
        const double2 a = Ax[t];
        r[t] = make_double2(b[t].x - zx.x - S.s * a.x, b[t].y - zx.y - S.s * a.y);
    }
}
// V0 = r / beta (0 where beta = 0 or the column is frozen)
__global__ void start_kernel(const double2 *__restrict__ r, double2 *V0, const double *beta, const int *active, i64 D, int nv,
                             int cw, int ry) {
    ROW_LOOP(D, nv, cw, ry) {
        const i64 t = mu * nv + c;
        const double bb = beta[c];
        V0[t] = (active[c] && bb > 0) ? make_double2(r[t].x / bb, r[t].y / bb) : make_double2(0, 0);
    }
}
// V_{j+1} = w / hn, as w * (1 / hn) with the reciprocal per column (ihn, from givens_kernel)
__global__ void normalize_kernel(double2 *w, const double *ihn, i64 D, int nv, int cw, int ry) {
    ROW_LOOP(D, nv, cw, ry) {
        const i64 t = mu * nv + c;
        const double r = ihn[c];
        w[t] = make_double2(w[t].x * r, w[t].y * r);
    }
}

// Per column: new Hessenberg column j (CGS coefficients hsum, subdiagonal sqrt(hn2)), previous rotations,
// new rotation, update g, count columns whose residual estimate is still above the target.
__global__ void givens_kernel(int j, int m, int nv, const double2 *hsum, int hld, const double *hn2, double2 *H, double2 *cs,
                              double2 *sn, double2 *g, const double *target, const int *active, double *res, int *nunconv,
                              double *ihn) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nv) return;
    double2 *Hc = H + (i64)c * (m + 1) * m;   // H[c][row][col], row < m+1, col < m
    for (int i = 0; i <= j; ++i) Hc[i * m + j] = hsum[(i64)c * hld + i];
    double hn = sqrt(hn2[c]);
    ihn[c] = hn > 1e-300 ? 1.0 / hn : 0.0;
    Hc[(j + 1) * m + j] = make_double2(hn, 0);
    double2 *csc = cs + (i64)c * m, *snc = sn + (i64)c * m, *gc = g + (i64)c * (m + 1);
    for (int i = 0; i < j; ++i) {
        double2 a = Hc[i * m + j], b = Hc[(i + 1) * m + j];
        double2 ci = csc[i], si = snc[i];
        // [conj(c) conj(s); -s c] [a; b]
        double2 na = make_double2(ci.x * a.x + ci.y * a.y + si.x * b.x + si.y * b.y, ci.x * a.y - ci.y * a.x + si.x * b.y - si.y * b.x);
        double2 nb = make_double2(-(si.x * a.x - si.y * a.y) + ci.x * b.x - ci.y * b.y, -(si.x * a.y + si.y * a.x) + ci.x * b.y + ci.y * b.x);
        Hc[i * m + j] = na;
        Hc[(i + 1) * m + j] = nb;
    }
    double2 a = Hc[j * m + j], b = Hc[(j + 1) * m + j];
    double den = sqrt(a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y);
    double2 cj = den > 0 ? make_double2(a.x / den, a.y / den) : make_double2(1, 0);
    double2 sj = den > 0 ? make_double2(b.x / den, b.y / den) : make_double2(0, 0);
    csc[j] = cj;
    snc[j] = sj;
    Hc[j * m + j] = make_double2(den, 0);
    Hc[(j + 1) * m + j] = make_double2(0, 0);
    double2 gj = gc[j];
    gc[j + 1] = make_double2(-(sj.x * gj.x - sj.y * gj.y), -(sj.x * gj.y + sj.y * gj.x));
    gc[j] = make_double2(cj.x * gj.x + cj.y * gj.y, cj.x * gj.y - cj.y * gj.x);
    double r = sqrt(gc[j + 1].x * gc[j + 1].x + gc[j + 1].y * gc[j + 1].y);
    res[c] = r;
    if (active[c] && r > target[c]) atomicAdd(nunconv, 1);
}

// y = H^-1 g (upper triangular, size J) then x += P (sum_i y_i V_i)
__global__ void trisolve_kernel(int J, int m, int nv, const double2 *H, const double2 *g, double2 *y) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nv) return;
    const double2 *Hc = H + (i64)c * (m + 1) * m;
    const double2 *gc = g + (i64)c * (m + 1);
    double2 *yc = y + (i64)c * m;
    for (int i = J - 1; i >= 0; --i) {
        double2 s = gc[i];
        for (int k = i + 1; k < J; ++k) {
            double2 p = cmul(Hc[i * m + k], yc[k]);
            s.x -= p.x;
            s.y -= p.y;
        }
        double2 d = Hc[i * m + i];
        double den = d.x * d.x + d.y * d.y;
        yc[i] = den > 0 ? cmul(s, cdiv1(d)) : make_double2(0, 0);
    }
}
__global__ void update_kernel(const double2 *__restrict__ P, int J, int m, const double2 *__restrict__ V, i64 vstride,
                              const double2 *__restrict__ y, double2 *x, i64 D, int nv, int cw, int ry) {
    ROW_LOOP(D, nv, cw, ry) {
        const i64 t = mu * nv + c;
        double2 acc = make_double2(0, 0);
        for (int i = 0; i < J; ++i) {
            const double2 p = cmul(y[(i64)c * m + i], V[(i64)i * vstride + t]);
            acc.x += p.x;
            acc.y += p.y;
        }
        const double2 u = cmul(P[t], acc);
        x[t].x += u.x;
        x[t].y += u.y;
    }
}
__global__ void init_cycle_kernel(int nv, int m, const double *beta2, double *beta, double2 *g, const double *target, int *active) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nv) return;
    double b = sqrt(beta2[c]);
    beta[c] = b;
    active[c] = b > target[c] ? 1 : 0;
    double2 *gc = g + (i64)c * (m + 1);
    for (int i = 0; i <= m; ++i) gc[i] = make_double2(0, 0);
    gc[0] = make_double2(active[c] ? b : 0.0, 0);
}
__global__ void scatter_g_kernel(int sector, const double2 *Ct, int N, int pend, int p0, int nw, int nv, double2 *G, int K,
                                 int w0, int nomega) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N * nv; t += gridDim.x * blockDim.x) {
        int row = t / nv, c = t % nv;
        int col_orb = p0 + c / nw, w = c % nw;
        if (col_orb >= pend) continue;
        int p, q;
        if (sector == CCGF_SECTOR_IP) { q = row; p = col_orb; }   // G-[p,q] = e_q . X_p
        else { p = row; q = col_orb; }                            // G+[p,q] = e_p . Y_q
        i64 gi = (((i64)K * nomega + w0 + w) * N + p) * N + q;
        G[gi].x += Ct[t].x;
        G[gi].y += Ct[t].y;
    }
}

// launch shape of ortho_dot_kernel: nv x ry threads (ry rows in flight per column, <= 256 threads),
// four blocks per SM, every block a contiguous range of rows
struct OrthoGrid {
    bool ok;   // false: nv > 256 (the atomic-reduction kernel runs instead)
    unsigned nblk, threads;
    int ry;
    i64 rpb;
    size_t smem;
};
inline OrthoGrid ortho_grid(i64 D, int nv) {
    OrthoGrid g{};
    g.ok = nv >= 1 && nv <= 256;
    g.ry = std::max(1, 256 / std::max(1, nv));
    g.threads = (unsigned)(nv * g.ry);
    const i64 want = 152 * 4;
    g.rpb = std::max<i64>(g.ry, ceil_div(D, want));
    g.nblk = (unsigned)ceil_div(D, g.rpb);
    g.smem = sizeof(double2) * 8 * (size_t)nv * g.ry;
    return g;
}

// launch shape of the ROW_LOOP kernels: columns cw = min(nv, 1024), ry rows so a block has about 256
// threads, eight blocks per SM (fewer for short arrays)
struct RowGrid {
    unsigned blocks, threads;
    int cw, ry;
};
inline RowGrid row_grid(i64 D, int nv) {
    RowGrid g{};
    g.cw = std::max(1, std::min(nv, 1024));
    g.ry = std::max(1, 256 / g.cw);
    g.threads = (unsigned)(g.cw * g.ry);
    g.blocks = (unsigned)std::max<i64>(1, std::min<i64>(ceil_div(D, g.ry), 152 * 8));
    return g;
}

inline unsigned g1(i64 n) {
    i64 g = ceil_div(n, 256);
    return (unsigned)std::max<i64>(1, std::min<i64>(g, 152 * 16));
}

// per column: mode 0 -> x0 = 0, r = b (cold); 1 -> keep (X, R); 2 -> (Xb, Rb)
__global__ void select_kernel(const int *mode, double2 *X, double2 *R, const double2 *Xb, const double2 *Rb, const double2 *B,
                              i64 D, int nv) {
    for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t < D * nv; t += (i64)gridDim.x * blockDim.x) {
        int md = mode[t % nv];
        if (md == 0) {
            X[t] = make_double2(0, 0);
            R[t] = B[t];
        } else if (md == 2) {
            X[t] = Xb[t];
            R[t] = Rb[t];
        }
    }
}

// cap[mu][p * ncw + w0 + w] = X[mu][(p - p0) * nw + w] for the batch's orbitals p < pend
__global__ void mor_copy_kernel(const double2 *__restrict__ X, i64 D, int nv, int p0, int pend, int nw, int w0, int N, int ncw,
                                double2 *cap) {
    for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t < D * nv; t += (i64)gridDim.x * blockDim.x) {
        const i64 mu = t / nv;
        const int c = (int)(t % nv), p = p0 + c / nw, w = c % nw;
        if (p < pend) cap[mu * ((i64)N * ncw) + (i64)p * ncw + w0 + w] = X[t];
    }
}

}  // namespace

void mor_capture_columns(ccgf_handle *h, const double2 *X, i64 D, int nv, int p0, int pend, int nw, int w0, cudaStream_t st) {
    mor_copy_kernel<<<g1(D * nv), 256, 0, st>>>(X, D, nv, p0, pend, nw, w0, h->n, h->mor_cap.nw, h->mor_cap.X);
    h->launches++;
}

void vcache_free(ccgf_handle *h) {
    for (auto *&vc : h->vcache) {
        delete vc;
        vc = nullptr;
    }
    h->vcache_bytes = 0;
}

ccgf_status diag_estimate_device(ccgf_handle *h, int sector, int K, double *d, cudaStream_t st) {
    const i64 D = sector == CCGF_SECTOR_IP ? h->dim_ip : h->dim_ea;
    diag_kernel<<<g1(D), 256, 0, st>>>(sector, K, h->nk, h->o, h->v, h->kadd_d.p, h->ksub_d.p, h->W[BUF_FOO].p,
                                       h->W[BUF_FVV].p, d, D);
    h->launches++;
    CCGF_CUDA_TRY(cudaGetLastError());
    return CCGF_OK;
}

ccgf_status solve_gf(ccgf_handle *h, int sectors, int nomega, const double *omega, double eta, const ccgf_options *opt,
                     double *G_out, int G_on_device, ccgf_stats *stats, cudaStream_t st) {
    const int nk = h->nk, N = h->n, o = h->o, v = h->v;
    const int kbeg = opt->kpoint >= 0 ? opt->kpoint : 0, kend = opt->kpoint >= 0 ? opt->kpoint + 1 : nk;
    const int pbeg = opt->orbital_count > 0 ? opt->orbital_first : 0;
    const int pend = opt->orbital_count > 0 ? opt->orbital_first + opt->orbital_count : N;
    const int NS = pend - pbeg;   // orbitals (right-hand sides per frequency) solved
    const int m_req = std::max(2, std::min(opt->restart_m, 128));
    int nwc = std::max(1, std::min(opt->omega_chunk, nomega));
    const double tol = opt->tol;
    const i64 Gn = (i64)nk * nomega * N * N;
    ccgf_stats S{};
    double warm_rel_sum = 0, warm_net_sum = 0, warm_base_sum = 0;
    i64 warm_count = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, es0 = nullptr, es1 = nullptr, ev2 = nullptr, er0 = nullptr, er1 = nullptr;
    bool refine_pending = false;   // er0 / er1 bracket an FP64 residual sigma not yet added to refine_ms
    int *nunconv_h = nullptr;
    auto cleanup = on_scope_exit([&] {
        if (nunconv_h) cudaFreeHost(nunconv_h);
        for (cudaEvent_t e : {ev0, ev1, es0, es1, ev2, er0, er1})
            if (e) cudaEventDestroy(e);
    });
    CCGF_CUDA_TRY(cudaEventCreate(&ev2));
    CCGF_CUDA_TRY(cudaEventCreate(&er0));
    CCGF_CUDA_TRY(cudaEventCreate(&er1));
    CCGF_CUDA_TRY(cudaEventCreate(&ev0));
    CCGF_CUDA_TRY(cudaEventCreate(&ev1));
    CCGF_CUDA_TRY(cudaEventCreate(&es0));
    CCGF_CUDA_TRY(cudaEventCreate(&es1));
    cudaEventRecord(ev0, st);
    const i64 launches0 = h->launches;

    DBuf<double2> Gd;
    double2 *G = nullptr;
    if (G_on_device) G = (double2 *)G_out;
    else {
        CCGF_TRY(dalloc(Gd, Gn));
        G = Gd.p;
    }
    CCGF_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(double2) * Gn, st));

    ccgf_status final_status = CCGF_OK;
    CCGF_CUDA_TRY(cudaMallocHost(&nunconv_h, sizeof(int)));
    double sigma_ms = 0;

    // Batch plan from the free device memory. Per column a batch holds the Krylov basis (m + 1
    // vectors), five work vectors, the preconditioner table and its share of the sigma scratch
    // (FP64, plus FP32 for a low-precision inner sigma). All orbitals x a frequency chunk form one batch when they fit;
    // otherwise the restart length shrinks (not below 10), then the orbitals are split into chunks
    // of equal width (the last one padded with zero columns, so every batch reuses one sigma plan),
    // then the frequency chunk shrinks. Low-precision copies of the intermediates are decided first,
    // leaving room for the smallest batch the largest sector needs.
    const i64 Dmax_s = (sectors & CCGF_SECTOR_EA) ? h->dim_ea : h->dim_ip;
    // low-precision inner sigma (iterative refinement); CCGF_FP64_TC counts as FP64
    const bool lowp = opt->prec == CCGF_FP32 || opt->prec == CCGF_TF32X3;
    // sigma of the true residual
    const ccgf_precision rprec = opt->prec == CCGF_FP64_TC ? CCGF_FP64_TC : (lowp ? opt->refine_prec : CCGF_FP64);
    auto column_bytes = [&](i64 D, int mm) -> double {
        const double scratch = (double)sigma_scratch_per_column(h) * (16.0 + (lowp ? 8.0 : 0.0)) + (lowp ? 8.0 * D : 0.0);
        return 16.0 * D * (mm + 7) + scratch + 16.0 * 304 * N;
    };
    {
        const int min_cols = std::min(NS * nwc, 16);
        // the sector loop's fixed share (right-hand / left vectors, a 4 GB margin) plus a small batch
        const double fixed = (double)(4ull << 30) + 32.0 * Dmax_s * N;
        const double reserve = fixed + column_bytes(Dmax_s, std::min(m_req, 20)) * min_cols + (double)(2ull << 30);
        size_t fr = 0, tot = 0;
        CCGF_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
        // copies made by earlier sigma calls (with a smaller reserve) give way to the solve's batch
        if ((double)fr < reserve) release_caches(h);
        if (lowp) CCGF_TRY(ensure_fp32(h, st, (size_t)reserve));
        if (opt->prec == CCGF_TF32X3) {
            if (!h->tc_err.p) {
                CCGF_TRY(dalloc(h->tc_err, 1));
                CCGF_CUDA_TRY(cudaMemsetAsync(h->tc_err.p, 0, sizeof(int), st));
            }
            CCGF_TRY(tc_prepare(h, st, (size_t)reserve));
        }
    }

    for (int sector = CCGF_SECTOR_IP; sector <= CCGF_SECTOR_EA; ++sector) {
        if (!(sectors & sector)) continue;
        const i64 D = sector == CCGF_SECTOR_IP ? h->dim_ip : h->dim_ea;
        const double s = sector == CCGF_SECTOR_IP ? 1.0 : -1.0;
        int m = m_req, np = NS;
        {
            size_t fr = 0, tot = 0;
            CCGF_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
            // minus the right-hand / left vectors and a margin for split-K partial sums and tables
            const double avail = (double)fr - (double)(4ull << 30) - 32.0 * D * N;
            auto fits = [&](int cols, int mm) { return column_bytes(D, mm) * cols <= avail; };
            while (!fits(NS * nwc, m) && m > 10) m = std::max(10, m - 5);
            if (!fits(NS * nwc, m)) {
                np = (int)std::max<double>(1.0, std::floor(avail / column_bytes(D, m) / nwc));
                np = std::min(np, NS);
                if (np < NS) np = (int)ceil_div(NS, ceil_div(NS, np));   // equal chunk widths
                if (!fits(np * nwc, m)) {
                    np = 1;
                    nwc = (int)std::max<double>(1.0, std::floor(avail / column_bytes(D, m)));
                }
            }
            if (!fits(np * nwc, m)) {
                set_last_error("not enough device memory for one right-hand side of this sector");
                return CCGF_ERR_OOM;
            }
        }
        S.restart_used = m;
        S.columns_per_batch = std::max<long long>(S.columns_per_batch, (long long)np * nwc);
        const int nvmax = np * nwc;
        DBuf<double2> Bq, E, B, X, R, U, AU, V, Ct, Hs, Hs2, Hm, cs, sn, g, y, z, Wk, Op;
        DBuf<double2> Pt;
        DBuf<double> dvec, beta2, beta, hn2, ihn, target, res;
        DBuf<int> active, nunconv;
        CCGF_TRY(dalloc(Bq, D * N));
        CCGF_TRY(dalloc(E, (i64)N * D));
        CCGF_TRY(dalloc(B, D * nvmax));
        CCGF_TRY(dalloc(X, D * nvmax));
        CCGF_TRY(dalloc(R, D * nvmax));
        CCGF_TRY(dalloc(U, D * nvmax));
        CCGF_TRY(dalloc(AU, D * nvmax));
        CCGF_TRY(dalloc(V, (i64)(m + 1) * D * nvmax));
        CCGF_TRY(dalloc(Ct, (i64)N * nvmax));
        CCGF_TRY(dalloc(Wk, (i64)304 * N * nvmax));
        CCGF_TRY(dalloc(Op, (i64)608 * (m + 1) * nvmax));   // CGS partial sums (ortho_grid: at most 608 blocks)
        CCGF_TRY(dalloc(Hs, (i64)nvmax * (m + 1)));
        CCGF_TRY(dalloc(Hs2, (i64)nvmax * (m + 1)));
        CCGF_TRY(dalloc(Hm, (i64)nvmax * (m + 1) * m));
        CCGF_TRY(dalloc(cs, (i64)nvmax * m));
        CCGF_TRY(dalloc(sn, (i64)nvmax * m));
        CCGF_TRY(dalloc(g, (i64)nvmax * (m + 1)));
        CCGF_TRY(dalloc(y, (i64)nvmax * m));
        CCGF_TRY(dalloc(z, nvmax));
        CCGF_TRY(dalloc(dvec, D));
        CCGF_TRY(dalloc(beta2, nvmax));
        CCGF_TRY(dalloc(beta, nvmax));
        CCGF_TRY(dalloc(hn2, nvmax));
        CCGF_TRY(dalloc(ihn, nvmax));
        CCGF_TRY(dalloc(Pt, D * nvmax));
        CCGF_TRY(dalloc(target, nvmax));
        CCGF_TRY(dalloc(res, nvmax));
        CCGF_TRY(dalloc(active, nvmax));
        CCGF_TRY(dalloc(nunconv, 1));
        auto free_all = [&]() {
            DBuf<double2> *zb[] = {&Bq, &E, &B, &X, &R, &U, &AU, &V, &Ct, &Hs, &Hs2, &Hm, &cs, &sn, &g, &y, &z, &Wk};
            for (auto *b : zb) dfree(*b);
            dfree(Pt);
            DBuf<double> *db[] = {&dvec, &beta2, &beta, &hn2, &ihn, &target, &res};
            for (auto *b : db) dfree(*b);
            dfree(active);
            dfree(nunconv);
        };
        for (int K = kbeg; K < kend; ++K) {
            const size_t vbytes = sizeof(double2) * (size_t)D * N;
            const int vkey = (sector - 1) * nk + K;
            if (h->vcache.empty()) h->vcache.assign(2 * nk, nullptr);
            if (ccgf_handle::VecCache *vc = h->vcache[vkey]) {
                CCGF_CUDA_TRY(cudaMemcpyAsync(Bq.p, vc->Bq.p, vbytes, cudaMemcpyDeviceToDevice, st));
                CCGF_CUDA_TRY(cudaMemcpyAsync(E.p, vc->E.p, vbytes, cudaMemcpyDeviceToDevice, st));
            } else {
                for (int p = 0; p < N; ++p) {
                    CCGF_TRY(make_rhs(h, sector, K, p, Bq.p + p, N, st));
                    CCGF_TRY(make_left(h, sector, K, p, E.p + (i64)p * D, 1, st));
                }
                // keep them for later solves while the cache stays below 2 GB and 2 % of the device
                size_t fr = 0, tot = 0;
                if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && h->vcache_bytes + 2 * vbytes <= std::min<size_t>((size_t)2 << 30, tot / 50) &&
                    fr > 2 * vbytes + ((size_t)4 << 30)) {
                    auto *nvc = new ccgf_handle::VecCache();
                    if (dalloc(nvc->Bq, D * N) == CCGF_OK && dalloc(nvc->E, D * N) == CCGF_OK) {
                        CCGF_CUDA_TRY(cudaMemcpyAsync(nvc->Bq.p, Bq.p, vbytes, cudaMemcpyDeviceToDevice, st));
                        CCGF_CUDA_TRY(cudaMemcpyAsync(nvc->E.p, E.p, vbytes, cudaMemcpyDeviceToDevice, st));
                        h->vcache[vkey] = nvc;
                        h->vcache_bytes += 2 * vbytes;
                    } else {
                        delete nvc;
                    }
                }
            }
            diag_kernel<<<g1(D), 256, 0, st>>>(sector, K, nk, o, v, h->kadd_d.p, h->ksub_d.p, h->W[BUF_FOO].p, h->W[BUF_FVV].p, dvec.p, D);
            h->launches++;
            for (int w0 = 0; w0 < nomega; w0 += nwc)
            for (int p0 = pbeg; p0 < pend; p0 += np) {
                const int nw = std::min(nwc, nomega - w0);
                const int nv = np * nw;
                const i64 Dn = D * nv;
                std::vector<double2> zh(nv);
                for (int c = 0; c < nv; ++c) zh[c] = make_double2(omega[w0 + c % nw], sector == CCGF_SECTOR_IP ? -eta : eta);
                CCGF_CUDA_TRY(cudaMemcpyAsync(z.p, zh.data(), sizeof(double2) * nv, cudaMemcpyHostToDevice, st));
                Shift Sh{z.p, s, dvec.p};
                const RowGrid rg = row_grid(D, nv);
                ptab_kernel<<<rg.blocks, rg.threads, 0, st>>>(Sh, Pt.p, D, nv, rg.cw, rg.ry);
                h->launches++;
                expand_kernel<<<g1(Dn), 256, 0, st>>>(Bq.p, B.p, D, N, pend, p0, nw, nv);
                h->launches++;
                CCGF_CUDA_TRY(cudaMemsetAsync(X.p, 0, sizeof(double2) * Dn, st));
                CCGF_CUDA_TRY(cudaMemcpyAsync(R.p, B.p, sizeof(double2) * Dn, cudaMemcpyDeviceToDevice, st));
                const i64 rpb = std::max<i64>(64, ceil_div(D, std::max<i64>(1, 2048 / (i64)ceil_div(nv, 32))));
                dim3 rgrid((unsigned)ceil_div(nv, 32), (unsigned)ceil_div(D, rpb));
                const OrthoGrid og = ortho_grid(D, nv);
                // target = tol * ||b||
                CCGF_CUDA_TRY(cudaMemsetAsync(beta2.p, 0, sizeof(double) * nv, st));
                colnorm2_kernel<<<rgrid, dim3(32, 8), 0, st>>>(B.p, beta2.p, D, nv, rpb);
                h->launches++;
                std::vector<double> b2(nv);
                CCGF_CUDA_TRY(cudaMemcpyAsync(b2.data(), beta2.p, sizeof(double) * nv, cudaMemcpyDeviceToHost, st));
                CCGF_CUDA_TRY(cudaStreamSynchronize(st));
                std::vector<double> tg(nv);
                for (int c = 0; c < nv; ++c) tg[c] = tol * std::sqrt(b2[c]);
                CCGF_CUDA_TRY(cudaMemcpyAsync(target.p, tg.data(), sizeof(double) * nv, cudaMemcpyHostToDevice, st));
                bool warm_lowp = false;   // R from the warm start's residual in the low-precision form
                if (opt->warm_start && np == N && NS == N) {
                    // learned initial vectors: per column keep the candidate (network, baseline, cold) with the
                    // smallest true residual; the cold start's residual is |b|
                    bool used = false, net = false;
                    CCGF_TRY(warmstart_infer(h, sector, K, omega + w0, nw, dvec.p, X.p, U.p, &used, &net, st));
                    if (used) {
                        auto resid2 = [&](const double2 *x, double2 *r, std::vector<double> &out) -> ccgf_status {
                            CCGF_TRY(sigma_apply(h, sector, K, nv, x, AU.p, opt->prec, st));
                            if (!lowp) S.fp64_sigma_calls++; else S.lowp_sigma_calls++;
                            residual_kernel<<<rg.blocks, rg.threads, 0, st>>>(Sh, B.p, x, AU.p, r, D, nv, rg.cw, rg.ry);
                            h->launches++;
                            CCGF_CUDA_TRY(cudaMemsetAsync(beta2.p, 0, sizeof(double) * nv, st));
                            colnorm2_kernel<<<rgrid, dim3(32, 8), 0, st>>>(r, beta2.p, D, nv, rpb);
                            h->launches++;
                            out.resize(nv);
                            CCGF_CUDA_TRY(cudaMemcpyAsync(out.data(), beta2.p, sizeof(double) * nv, cudaMemcpyDeviceToHost, st));
                            CCGF_CUDA_TRY(cudaStreamSynchronize(st));
                            return CCGF_OK;
                        };
                        std::vector<double> rn, rb;
                        CCGF_TRY(resid2(X.p, R.p, rn));
                        if (net) CCGF_TRY(resid2(U.p, V.p, rb));     // baseline candidate (V slot 0 is free here)
                        std::vector<int> mode(nv);                     // 0 cold, 1 network / baseline-only, 2 baseline
                        for (int c = 0; c < nv; ++c) {
                            double best = b2[c];
                            mode[c] = 0;
                            if (rn[c] < best) { best = rn[c]; mode[c] = 1; }
                            if (net && rb[c] < best) { best = rb[c]; mode[c] = 2; }
                            S.warm_columns += mode[c] ? 1 : 0;
                            S.warm_fallbacks += mode[c] ? 0 : 1;
                            if (b2[c] > 0) {
                                warm_rel_sum += std::sqrt(best / b2[c]);
                                if (net) {
                                    warm_net_sum += std::sqrt(rn[c] / b2[c]);
                                    warm_base_sum += std::sqrt(rb[c] / b2[c]);
                                } else {
                                    warm_base_sum += std::sqrt(rn[c] / b2[c]);
                                }
                                warm_count++;
                            }
                        }
                        CCGF_CUDA_TRY(cudaMemcpyAsync(active.p, mode.data(), sizeof(int) * nv, cudaMemcpyHostToDevice, st));
                        select_kernel<<<g1(Dn), 256, 0, st>>>(active.p, X.p, R.p, U.p, V.p, B.p, D, nv);
                        h->launches++;
                        warm_lowp = lowp;
                    }
                }
                i64 it_total = 0;
                int cycles = 0;
                bool converged = false;
                double maxres = 0;
                // R holds the FP64 true residual (else the residual of the low-precision operator: a GMRES
                // restart that had not met the target yet)
                bool r_fp64 = !warm_lowp;
                bool tightened = false;
                std::vector<double> tg_inner(nv);
                auto true_residual = [&]() -> ccgf_status {
                    cudaEventRecord(er0, st);
                    CCGF_TRY(sigma_apply(h, sector, K, nv, X.p, AU.p, rprec, st));
                    cudaEventRecord(er1, st);
                    refine_pending = true;
                    S.fp64_sigma_calls++;
                    residual_kernel<<<rg.blocks, rg.threads, 0, st>>>(Sh, B.p, X.p, AU.p, R.p, D, nv, rg.cw, rg.ry);
                    h->launches++;
                    r_fp64 = true;
                    return CCGF_OK;
                };
                for (;;) {
                    // beta = ||r||, freeze columns already below target
                    CCGF_CUDA_TRY(cudaMemsetAsync(beta2.p, 0, sizeof(double) * nv, st));
                    colnorm2_kernel<<<rgrid, dim3(32, 8), 0, st>>>(R.p, beta2.p, D, nv, rpb);
                    h->launches++;
                    init_cycle_kernel<<<(unsigned)ceil_div(nv, 128), 128, 0, st>>>(nv, m, beta2.p, beta.p, g.p, target.p, active.p);
                    h->launches++;
                    std::vector<double> bh(nv);
                    CCGF_CUDA_TRY(cudaMemcpyAsync(bh.data(), beta.p, sizeof(double) * nv, cudaMemcpyDeviceToHost, st));
                    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
                    if (refine_pending) {
                        float rms = 0;
                        cudaEventElapsedTime(&rms, er0, er1);
                        S.refine_ms += rms;
                        refine_pending = false;
                    }
                    int nact = 0;
                    maxres = 0;
                    for (int c = 0; c < nv; ++c) {
                        double bn = tg[c] / tol;
                        double rr = bn > 0 ? bh[c] / bn : 0.0;
                        maxres = std::max(maxres, rr);
                        if (bh[c] > tg[c]) nact++;
                    }
                    const bool stop = nact == 0 || cycles >= opt->max_refine || it_total >= opt->max_iter;
                    if (stop && !r_fp64) {
                        // decide (and report) on the FP64 true residual only
                        CCGF_TRY(true_residual());
                        continue;
                    }
                    if (nact == 0) { converged = true; break; }
                    if (stop) break;
                    if (lowp && r_fp64 && cycles > 0 && !tightened) {
                        // the FP64 check failed after a low-precision iteration that had met the target:
                        // from here on that iteration aims a decade lower, so that the next check is not
                        // decided by the low-precision operator's rounding (one refinement step instead
                        // of many that each gain little)
                        for (int c = 0; c < nv; ++c) tg_inner[c] = 0.1 * tg[c];
                        CCGF_CUDA_TRY(cudaMemcpyAsync(target.p, tg_inner.data(), sizeof(double) * nv, cudaMemcpyHostToDevice, st));
                        tightened = true;
                        continue;
                    }
                    cycles++;
                    start_kernel<<<rg.blocks, rg.threads, 0, st>>>(R.p, V.p, beta.p, active.p, D, nv, rg.cw, rg.ry);
                    h->launches++;
                    int J = 0;
                    for (int j = 0; j < m; ++j) {
                        double2 *Vj = V.p + (i64)j * Dn, *Vn = V.p + (i64)(j + 1) * Dn;
                        precond_kernel<<<rg.blocks, rg.threads, 0, st>>>(Pt.p, Vj, U.p, D, nv, rg.cw, rg.ry);
                        h->launches++;
                        cudaEventRecord(es0, st);
                        CCGF_TRY(sigma_apply(h, sector, K, nv, U.p, AU.p, opt->prec, st));
                        cudaEventRecord(es1, st);
                        if (!lowp) S.fp64_sigma_calls++; else S.lowp_sigma_calls++;
                        shift_kernel<<<rg.blocks, rg.threads, 0, st>>>(Sh, U.p, AU.p, Vn, D, nv, rg.cw, rg.ry);
                        h->launches++;
                        for (int pass = 0; pass < 2; ++pass) {
                            // CGS2: pass 1 writes the coefficients into Hs, pass 2 into Hs2 and adds them to Hs;
                            // each pass subtracts its own projection
                            DBuf<double2> &hp = pass == 0 ? Hs : Hs2;
                            if (og.ok) {
                                ortho_dot_kernel<<<og.nblk, og.threads, og.smem, st>>>(V.p, Dn, Vn, Op.p, j + 1, D, nv, og.ry,
                                                                                    og.rpb);
                                ortho_sum_kernel<<<(unsigned)ceil_div((i64)(j + 1) * nv, 8), 256, 0, st>>>(Op.p, og.nblk, hp.p, m + 1, j + 1,
                                                                                                     nv, 0);
                                h->launches += 2;
                            } else {
                                CCGF_CUDA_TRY(cudaMemsetAsync(hp.p, 0, sizeof(double2) * nv * (m + 1), st));
                                cgs_dot_kernel<<<rgrid, dim3(32, 8), 0, st>>>(V.p, Dn, Vn, hp.p, m + 1, j + 1, D, nv, rpb);
                                h->launches++;
                            }
                            cgs_axpy_kernel<<<rg.blocks, rg.threads, 0, st>>>(V.p, Dn, Vn, hp.p, m + 1, j + 1, D, nv, rg.cw, rg.ry);
                            h->launches++;
                            if (pass == 1) {
                                // Hs += Hs2
                                PermDesc pd{};
                                pd.nd = 1;
                                pd.dims[0] = (i64)nv * (m + 1);
                                pd.sA[0] = 1;
                                pd.sC[0] = 1;
                                pd.total = pd.dims[0];
                                pd.batch = 1;
                                pd.offA = h->zero_tab.p;
                                pd.offC = h->zero_tab.p;
                                pd.alpha = make_double2(1, 0);
                                pd.beta = make_double2(1, 0);
                                h->launches += launch_zpermute<double>(pd, Hs2.p, Hs.p, st);
                            }
                        }
                        CCGF_CUDA_TRY(cudaMemsetAsync(hn2.p, 0, sizeof(double) * nv, st));
                        colnorm2_kernel<<<rgrid, dim3(32, 8), 0, st>>>(Vn, hn2.p, D, nv, rpb);
                        h->launches++;
                        CCGF_CUDA_TRY(cudaMemsetAsync(nunconv.p, 0, sizeof(int), st));
                        givens_kernel<<<(unsigned)ceil_div(nv, 128), 128, 0, st>>>(j, m, nv, Hs.p, m + 1, hn2.p, Hm.p, cs.p, sn.p, g.p,
                                                                                   target.p, active.p, res.p, nunconv.p, ihn.p);
                        h->launches++;
                        normalize_kernel<<<rg.blocks, rg.threads, 0, st>>>(Vn, ihn.p, D, nv, rg.cw, rg.ry);
                        h->launches++;
                        cudaEventRecord(ev2, st);
                        CCGF_CUDA_TRY(cudaMemcpyAsync(nunconv_h, nunconv.p, sizeof(int), cudaMemcpyDeviceToHost, st));
                        CCGF_CUDA_TRY(cudaStreamSynchronize(st));
                        float ms = 0, vms = 0;
                        cudaEventElapsedTime(&ms, es0, es1);
                        cudaEventElapsedTime(&vms, es1, ev2);
                        sigma_ms += ms;
                        // vector steps after the sigma: shift (3 vectors), two CGS passes (2 (J + 1) read
                        // + 1 written each, twice), norm (1), normalisation (2) with J = j + 1 basis vectors
                        S.vector_ms += vms;
                        S.vector_bytes += 16.0 * (double)Dn * (4.0 * (j + 1) + 12.0);
                        S.vector_flops += (double)Dn * (32.0 * (j + 1) + 14.0);
                        J = j + 1;
                        it_total++;
                        // stop the cycle a little below the target so the FP64 check passes
                        if (*nunconv_h == 0 || it_total >= opt->max_iter) break;
                    }
                    trisolve_kernel<<<(unsigned)ceil_div(nv, 128), 128, 0, st>>>(J, m, nv, Hm.p, g.p, y.p);
                    h->launches++;
                    update_kernel<<<rg.blocks, rg.threads, 0, st>>>(Pt.p, J, m, V.p, Dn, y.p, X.p, D, nv, rg.cw, rg.ry);
                    h->launches++;
                    if (lowp && *nunconv_h != 0) {
                        // the cycle ended at the restart length short of the target: restart from the
                        // residual of the low-precision operator; the FP64 residual is taken once the
                        // low-precision iteration meets the target (refinement step)
                        CCGF_TRY(sigma_apply(h, sector, K, nv, X.p, AU.p, opt->prec, st));
                        S.lowp_sigma_calls++;
                        residual_kernel<<<rg.blocks, rg.threads, 0, st>>>(Sh, B.p, X.p, AU.p, R.p, D, nv, rg.cw, rg.ry);
                        h->launches++;
                        r_fp64 = false;
                    } else {
                        CCGF_TRY(true_residual());
                    }
                }
                if (h->ws_capturing && np == N && NS == N) CCGF_TRY(warmstart_capture(h, sector, K, X.p, D, nw, w0, b2.data(), st));
                if (h->mor_cap.X && h->mor_cap.sector == sector && h->mor_cap.K == K)
                    mor_capture_columns(h, X.p, D, nv, p0, pend, nw, w0, st);
                S.inner_iterations += it_total;
                S.rhs_solved += (long long)std::min(np, pend - p0) * nw;
                S.max_rel_residual = std::max(S.max_rel_residual, maxres);
                if (!converged) final_status = CCGF_NOT_CONVERGED;
                // G contraction: Ct[q][c] = sum_mu E[q][mu] X[mu][c]
                {
                    GemmDesc gd{};
                    gd.M = N;
                    gd.N = nv;
                    gd.K = (int)D;
                    gd.nred = 1;
                    gd.batch = 1;
                    gd.rsA = D;
                    gd.csA = 1;
                    gd.rsB = nv;
                    gd.csB = 1;
                    gd.rsC = nv;
                    gd.csC = 1;
                    gd.offA = h->zero_tab.p;
                    gd.offB = h->zero_tab.p + 1;
                    gd.offC = h->zero_tab.p + 2;
                    gd.alpha = make_double2(1, 0);
                    gd.beta = make_double2(0, 0);
                    h->launches += launch_zgemm<double>(gd, E.p, X.p, Ct.p, st, Wk.p, Wk.n);
                    scatter_g_kernel<<<g1((i64)N * nv), 256, 0, st>>>(sector, Ct.p, N, pend, p0, nw, nv, G, K, w0, nomega);
                    h->launches++;
                }
                CCGF_CUDA_TRY(cudaGetLastError());
            }
        }
        CCGF_CUDA_TRY(cudaStreamSynchronize(st));
        free_all();
    }
    if (!G_on_device) CCGF_CUDA_TRY(cudaMemcpyAsync(G_out, G, sizeof(double2) * Gn, cudaMemcpyDeviceToHost, st));
    cudaEventRecord(ev1, st);
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    float tms = 0;
    cudaEventElapsedTime(&tms, ev0, ev1);
    S.total_ms = tms;
    if (warm_count > 0) {
        S.warm_rel_residual = warm_rel_sum / warm_count;
        S.warm_rel_residual_net = warm_net_sum / warm_count;
        S.warm_rel_residual_base = warm_base_sum / warm_count;
    }
    S.sigma_ms = sigma_ms;
    S.kernel_launches = h->launches - launches0;
    if (stats) *stats = S;
    dfree(Gd);
    if (opt->prec == CCGF_TF32X3 || rprec == CCGF_FP64_TC) CCGF_TRY(tc_error_check(h, st));
    return final_status;
}
