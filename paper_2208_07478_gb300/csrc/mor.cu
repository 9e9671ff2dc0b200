// Model-order-reduction CCGF (the paper's MOR paragraph): G on a full frequency grid from a reduced
// model built out of the solutions at a few model frequencies.
//
// For each sector and total momentum K:
//   1. the shifted systems of Eq. 6 are solved at the n_mor model frequencies for every orbital (the
//      batched GMRES of solve.cu, whose converged columns are captured: S = [X_p(w_i)], D x (nmo n_mor));
//   2. an orthonormal basis V of span(S): the Gram matrix S^H S is diagonalised (Jacobi, host, size
//      nmo n_mor), V = S U L^-1/2 over eigenvalues above 1e-14 of the largest (singular values above
//      1e-7 of the largest); a second pass on V^H V restores orthonormality to rounding;
//   3. the projected operator A_r = V^H (A V) (A V by the sigma kernels, in column chunks of the solve's
//      plan width), right-hand sides b_r = V^H b_p and left vectors e_r = e_q V;
//   4. for every grid frequency the reduced system (z + s A_r) y = b_r (dimension rank V) is solved by
//      LU with partial pivoting on the host and contracted into G (Eq. 7), G = G+ + G- (Eq. 9).
// The large products (Gram matrices, the basis, the projections) are GEMMs on the device.
#include "ccgf_internal.h"
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace {

typedef std::complex<double> cd;

__global__ void conj_copy_kernel(const double2 *__restrict__ a, double2 *__restrict__ b, i64 n) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) b[i] = make_double2(a[i].x, -a[i].y);
}
// dst[mu][c] = src[mu][c0 + c] for c < ncopy, 0 for ncopy <= c < nv (a column chunk of a [D][ld] array)
__global__ void chunk_in_kernel(const double2 *__restrict__ src, i64 D, int ld, int c0, int ncopy, int nv, double2 *dst) {
    for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t < D * nv; t += (i64)gridDim.x * blockDim.x) {
        const i64 mu = t / nv;
        const int c = (int)(t % nv);
        dst[t] = c < ncopy ? src[mu * ld + c0 + c] : make_double2(0.0, 0.0);
    }
}
__global__ void chunk_out_kernel(const double2 *__restrict__ src, i64 D, int nv, int ncopy, int ld, int c0, double2 *dst) {
    for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t < D * ncopy; t += (i64)gridDim.x * blockDim.x) {
        const i64 mu = t / ncopy;
        const int c = (int)(t % ncopy);
        dst[mu * ld + c0 + c] = src[mu * nv + c];
    }
}
inline unsigned gs(i64 n) {
    i64 g = ceil_div(n, 256);
    return (unsigned)std::max<i64>(1, std::min<i64>(g, 152 * 16));
}

// C[M x N] = A[M x K] B[K x N], row-major with leading dimensions, FP64 complex on the device
ccgf_status dgemm(ccgf_handle *h, int M, int N, int K, const double2 *A, i64 rsA, i64 csA, const double2 *B, i64 rsB, i64 csB,
                  double2 *C, i64 rsC, DBuf<double2> &work, cudaStream_t st) {
    GemmDesc g{};
    g.M = M;
    g.N = N;
    g.K = K;
    g.nred = 1;
    g.batch = 1;
    g.rsA = rsA;
    g.csA = csA;
    g.rsB = rsB;
    g.csB = csB;
    g.rsC = rsC;
    g.csC = 1;
    g.offA = h->zero_tab.p;
    g.offB = h->zero_tab.p + 1;
    g.offC = h->zero_tab.p + 2;
    g.alpha = make_double2(1, 0);
    g.beta = make_double2(0, 0);
    const i64 need = zgemm_workspace_elems(g);
    if (work.n < need) CCGF_TRY(dalloc(work, need));
    h->launches += launch_zgemm<double>(g, A, B, C, st, work.p, work.n);
    CCGF_CUDA_TRY(cudaGetLastError());
    return CCGF_OK;
}

// cyclic Jacobi diagonalisation of a Hermitian n x n matrix a (row-major, destroyed): eigenvalues w,
// eigenvectors as the columns of u
void jacobi_hermitian(std::vector<cd> &a, int n, std::vector<double> &w, std::vector<cd> &u) {
    u.assign((size_t)n * n, cd(0, 0));
    for (int i = 0; i < n; ++i) u[(size_t)i * n + i] = 1.0;
    auto A = [&](int i, int j) -> cd & { return a[(size_t)i * n + j]; };
    double norm = 0;
    for (auto &x : a) norm += std::norm(x);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += std::norm(A(i, j));
        if (off <= 1e-30 * norm) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                const cd b = A(p, q);
                const double ab = std::abs(b);
                if (ab <= 1e-300) continue;
                // D = diag(1, e^{-i phi}) makes the 2 x 2 block real, then a real rotation zeroes it
                const cd ph = b / ab;
                const double app = A(p, p).real(), aqq = A(q, q).real();
                const double tau = (aqq - app) / (2 * ab);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
                const double c = 1 / std::sqrt(1 + t * t), s = t * c;
                // column update: U = D R with R = [[c, s], [-s, c]]: col p' = c col_p - s conj(ph) col_q,
                //                col q' = s col_p + c conj(ph) col_q
                const cd cp = std::conj(ph);
                for (int k = 0; k < n; ++k) {
                    const cd akp = A(k, p), akq = A(k, q);
                    A(k, p) = c * akp - s * cp * akq;
                    A(k, q) = s * akp + c * cp * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const cd apk = A(p, k), aqk = A(q, k);
                    A(p, k) = c * apk - s * ph * aqk;
                    A(q, k) = s * apk + c * ph * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const cd ukp = u[(size_t)k * n + p], ukq = u[(size_t)k * n + q];
                    u[(size_t)k * n + p] = c * ukp - s * cp * ukq;
                    u[(size_t)k * n + q] = s * ukp + c * cp * ukq;
                }
                A(p, q) = 0;
                A(q, p) = 0;
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A(i, i).real();
}

// W = U_keep diag(lambda^-1/2) (n x r) for eigenvalues above rel * max; returns r
int whitening(const std::vector<cd> &gram, int n, double rel, std::vector<cd> &W) {
    std::vector<cd> a = gram, u;
    std::vector<double> w;
    jacobi_hermitian(a, n, w, u);
    double wmax = 0;
    for (double x : w) wmax = std::max(wmax, x);
    std::vector<int> keep;
    for (int i = 0; i < n; ++i)
        if (w[i] > rel * wmax && w[i] > 0) keep.push_back(i);
    const int r = (int)keep.size();
    W.assign((size_t)n * r, cd(0, 0));
    for (int j = 0; j < r; ++j) {
        const double sc = 1 / std::sqrt(w[keep[j]]);
        for (int i = 0; i < n; ++i) W[(size_t)i * r + j] = u[(size_t)i * n + keep[j]] * sc;
    }
    return r;
}

// solves M X = B (n x n, n x m, row-major) by LU with partial pivoting; false if singular
bool lu_solve(std::vector<cd> M, int n, std::vector<cd> &B, int m) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = std::abs(M[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (std::abs(M[(size_t)i * n + k]) > best) { best = std::abs(M[(size_t)i * n + k]); p = i; }
        if (!(best > 0)) return false;
        if (p != k) {
            for (int j = 0; j < n; ++j) std::swap(M[(size_t)k * n + j], M[(size_t)p * n + j]);
            for (int j = 0; j < m; ++j) std::swap(B[(size_t)k * m + j], B[(size_t)p * m + j]);
        }
        const cd d = M[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            const cd f = M[(size_t)i * n + k] / d;
            if (f == cd(0, 0)) continue;
            for (int j = k; j < n; ++j) M[(size_t)i * n + j] -= f * M[(size_t)k * n + j];
            for (int j = 0; j < m; ++j) B[(size_t)i * m + j] -= f * B[(size_t)k * m + j];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        const cd d = M[(size_t)k * n + k];
        for (int j = 0; j < m; ++j) {
            cd acc = B[(size_t)k * m + j];
            for (int i = k + 1; i < n; ++i) acc -= M[(size_t)k * n + i] * B[(size_t)i * m + j];
            B[(size_t)k * m + j] = acc / d;
        }
    }
    return true;
}

ccgf_status to_host(std::vector<cd> &out, const double2 *d, i64 n, cudaStream_t st) {
    out.resize(n);
    CCGF_CUDA_TRY(cudaMemcpyAsync(out.data(), d, sizeof(double2) * n, cudaMemcpyDeviceToHost, st));
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    return CCGF_OK;
}
ccgf_status to_dev(DBuf<double2> &d, const std::vector<cd> &in, cudaStream_t st) {
    CCGF_TRY(dalloc(d, (i64)in.size()));
    CCGF_CUDA_TRY(cudaMemcpyAsync(d.p, in.data(), sizeof(double2) * in.size(), cudaMemcpyHostToDevice, st));
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    return CCGF_OK;
}

// V^H S for device V [D][r], S [D][c]: conj(V)^T S, (r x c) on the host
ccgf_status project(ccgf_handle *h, const double2 *Vc, int r, const double2 *S, int c, i64 D, std::vector<cd> &out, DBuf<double2> &work,
                    cudaStream_t st) {
    DBuf<double2> P;
    CCGF_TRY(dalloc(P, (i64)r * c));
    CCGF_TRY(dgemm(h, r, c, (int)D, Vc, 1, r, S, c, 1, P.p, c, work, st));
    return to_host(out, P.p, (i64)r * c, st);
}

}  // namespace

ccgf_status solve_gf_mor(ccgf_handle *h, int sectors, int n_mor, const double *omega_mor, int nomega, const double *omega,
                         double eta, const ccgf_options *opt, double *G_out, int G_on_device, ccgf_stats *stats, cudaStream_t st) {
    const int nk = h->nk, N = h->n;
    const int kbeg = opt->kpoint >= 0 ? opt->kpoint : 0, kend = opt->kpoint >= 0 ? opt->kpoint + 1 : nk;
    const i64 Gn = (i64)nk * nomega * N * N;
    std::vector<cd> G((size_t)Gn, cd(0, 0));
    ccgf_stats S{}, Ssolve{};
    ccgf_options o = *opt;
    o.orbital_first = 0;
    o.orbital_count = 0;
    o.warm_start = 0;
    DBuf<double2> Gtmp, work;
    CCGF_TRY(dalloc(Gtmp, (i64)nk * n_mor * N * N));
    long long rank_max = 0;
    for (int sector = CCGF_SECTOR_IP; sector <= CCGF_SECTOR_EA; ++sector) {
        if (!(sectors & sector)) continue;
        const i64 D = sector == CCGF_SECTOR_IP ? h->dim_ip : h->dim_ea;
        const int C = N * n_mor;
        const double sgn = sector == CCGF_SECTOR_IP ? 1.0 : -1.0;
        for (int K = kbeg; K < kend; ++K) {
            // 1. solutions at the model frequencies
            DBuf<double2> Sx;
            CCGF_TRY(dalloc(Sx, D * C));
            h->mor_cap.sector = sector;
            h->mor_cap.K = K;
            h->mor_cap.nw = n_mor;
            h->mor_cap.X = Sx.p;
            o.kpoint = K;
            ccgf_status s = solve_gf(h, sector, n_mor, omega_mor, eta, &o, (double *)Gtmp.p, 1, &Ssolve, st);
            h->mor_cap.X = nullptr;
            if (s != CCGF_OK && s != CCGF_NOT_CONVERGED) return s;
            S.rhs_solved += Ssolve.rhs_solved;
            S.inner_iterations += Ssolve.inner_iterations;
            S.fp64_sigma_calls += Ssolve.fp64_sigma_calls;
            S.lowp_sigma_calls += Ssolve.lowp_sigma_calls;
            S.max_rel_residual = std::max(S.max_rel_residual, Ssolve.max_rel_residual);
            // 2. orthonormal basis: V1 = S W1, then V = V1 W2 (two Gram passes)
            DBuf<double2> Sc, Vb;
            CCGF_TRY(dalloc(Sc, D * C));
            conj_copy_kernel<<<gs(D * C), 256, 0, st>>>(Sx.p, Sc.p, D * C);
            h->launches++;
            std::vector<cd> gram, W1, W2;
            CCGF_TRY(project(h, Sc.p, C, Sx.p, C, D, gram, work, st));   // (S^H S)[i][j] with conj(S) as [D][C]
            const int r1 = whitening(gram, C, 1e-14, W1);
            if (r1 == 0) continue;
            DBuf<double2> W1d, V1;
            CCGF_TRY(to_dev(W1d, W1, st));
            CCGF_TRY(dalloc(V1, D * r1));
            CCGF_TRY(dgemm(h, (int)D, r1, C, Sx.p, C, 1, W1d.p, r1, 1, V1.p, r1, work, st));
            dfree(Sx);
            CCGF_TRY(dalloc(Sc, D * r1));
            conj_copy_kernel<<<gs(D * r1), 256, 0, st>>>(V1.p, Sc.p, D * r1);
            h->launches++;
            CCGF_TRY(project(h, Sc.p, r1, V1.p, r1, D, gram, work, st));
            const int r = whitening(gram, r1, 1e-14, W2);
            DBuf<double2> W2d;
            CCGF_TRY(to_dev(W2d, W2, st));
            CCGF_TRY(dalloc(Vb, D * r));
            CCGF_TRY(dgemm(h, (int)D, r, r1, V1.p, r1, 1, W2d.p, r, 1, Vb.p, r, work, st));
            dfree(V1);
            rank_max = std::max<long long>(rank_max, r);
            // 3. A V in column chunks of nmo (the plan width of the model solves), then the projections
            DBuf<double2> AV, xin, yout, Bq, E;
            CCGF_TRY(dalloc(AV, D * r));
            CCGF_TRY(dalloc(xin, D * N));
            CCGF_TRY(dalloc(yout, D * N));
            for (int c0 = 0; c0 < r; c0 += N) {
                const int nc = std::min(N, r - c0);
                chunk_in_kernel<<<gs(D * N), 256, 0, st>>>(Vb.p, D, r, c0, nc, N, xin.p);
                CCGF_TRY(sigma_apply(h, sector, K, N, xin.p, yout.p, CCGF_FP64, st));
                chunk_out_kernel<<<gs(D * nc), 256, 0, st>>>(yout.p, D, N, nc, r, c0, AV.p);
                h->launches += 2;
            }
            CCGF_TRY(dalloc(Bq, D * N));
            CCGF_TRY(dalloc(E, (i64)N * D));
            for (int p = 0; p < N; ++p) {
                CCGF_TRY(make_rhs(h, sector, K, p, Bq.p + p, N, st));
                CCGF_TRY(make_left(h, sector, K, p, E.p + (i64)p * D, 1, st));
            }
            CCGF_TRY(dalloc(Sc, D * r));
            conj_copy_kernel<<<gs(D * r), 256, 0, st>>>(Vb.p, Sc.p, D * r);
            h->launches++;
            std::vector<cd> Ar, Br, Er;
            CCGF_TRY(project(h, Sc.p, r, AV.p, r, D, Ar, work, st));
            CCGF_TRY(project(h, Sc.p, r, Bq.p, N, D, Br, work, st));
            {
                DBuf<double2> P;
                CCGF_TRY(dalloc(P, (i64)N * r));
                CCGF_TRY(dgemm(h, N, r, (int)D, E.p, D, 1, Vb.p, r, 1, P.p, r, work, st));
                CCGF_TRY(to_host(Er, P.p, (i64)N * r, st));
            }
            // 4. reduced systems on the grid: IP (w - i eta + A_r) y = b_r, EA (w + i eta - A_r) y = b_r
            for (int w = 0; w < nomega; ++w) {
                const cd z(omega[w], sector == CCGF_SECTOR_IP ? -eta : eta);
                std::vector<cd> M((size_t)r * r), Y = Br;
                for (int i = 0; i < r; ++i)
                    for (int j = 0; j < r; ++j) M[(size_t)i * r + j] = sgn * Ar[(size_t)i * r + j] + (i == j ? z : cd(0, 0));
                if (!lu_solve(M, r, Y, N)) {
                    set_last_error("model-order reduction: a reduced system is singular");
                    return CCGF_ERR_INVALID_ARG;
                }
                for (int q = 0; q < N; ++q)
                    for (int p = 0; p < N; ++p) {
                        cd acc(0, 0);
                        for (int i = 0; i < r; ++i) acc += Er[(size_t)q * r + i] * Y[(size_t)i * N + p];
                        // IP: G-[p,q] = e_q . X_p;  EA: G+[q,p] = e_q . Y_p
                        const i64 gi = sector == CCGF_SECTOR_IP ? (((i64)K * nomega + w) * N + p) * N + q
                                                                : (((i64)K * nomega + w) * N + q) * N + p;
                        G[(size_t)gi] += acc;
                    }
            }
        }
    }
    CCGF_CUDA_TRY(cudaMemcpyAsync(G_out, G.data(), sizeof(double2) * Gn, G_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost,
                                  st));
    CCGF_CUDA_TRY(cudaStreamSynchronize(st));
    S.columns_per_batch = rank_max;   // here: the largest reduced-model dimension
    if (stats) *stats = S;
    return CCGF_OK;
}
