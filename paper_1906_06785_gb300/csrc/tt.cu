// Tensor trains on the device (Section 4.1): storage, concatenation (vector
// addition), truncation T_eps and inner products.
//
// Truncation.  The paper's T_eps is the TT-SVD of Algorithm 4.1 applied to a
// train: orthogonalise right to left, then truncate left to right with
// delta = eps ||z|| / sqrt 2.  Here the orthogonalisation only forms R
// factors (R3 of z3^T, then R of the right unfolding of z2 x3 R3), which gives
// the singular values and left singular vectors of both unfoldings; the new
// cores are then obtained by projecting the ORIGINAL cores onto the kept left
// singular frames (P1 = U1^T z1, C2 = P1 x1 z2, new z3 = (U2^T C2) z3).  In
// exact arithmetic this is the same T_eps, and it needs no orthogonal factor Q.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <exception>
#include <thread>

#include "tt.cuh"

namespace tt {

tt_t* tt_alloc(tt_ctx* c, int n_t, int n_xi, int n_x, int r1, int r2, int cap1, int cap2) {
    TT_REQUIRE(n_t > 0 && n_xi > 0 && n_x > 0 && r1 > 0 && r2 > 0,
               "bad train shape %d %d %d ranks %d %d", n_t, n_xi, n_x, r1, r2);
    if (cap1 <= 0) cap1 = r1;
    if (cap2 <= 0) cap2 = r2;
    TT_REQUIRE(cap1 >= r1 && cap2 >= r2, "rank capacities (%d, %d) below the ranks (%d, %d)", cap1, cap2, r1, r2);
    // cores packed with the current ranks at offsets fixed by the capacities
    const size_t s1 = (size_t)n_t * cap1, s2 = (size_t)cap1 * n_xi * cap2, s3 = (size_t)n_x * cap2;
    tt_t* t = new tt_t;
    t->ctx = c;
    t->n_t = n_t; t->n_xi = n_xi; t->n_x = n_x; t->r1 = r1; t->r2 = r2;
    t->cap1 = cap1; t->cap2 = cap2;
    t->bytes = (s1 + s2 + s3) * sizeof(double);
    try {
        t->base = static_cast<double*>(ctx_malloc(c, t->bytes));
    } catch (...) {
        delete t;
        throw;
    }
    t->z1 = t->base;
    t->z2 = t->base + s1;
    t->z3 = t->base + s1 + s2;
    return t;
}

void tt_free(tt_t* t) {
    if (!t) return;
    if (t->base) ctx_free(t->ctx, t->base, t->bytes);
    delete t;
}

TTPtr zeros(tt_ctx* c, int n_t, int n_xi, int n_x) {
    TTPtr t = wrap(tt_alloc(c, n_t, n_xi, n_x, 1, 1));
    fill_zero(c, t->base, (size_t)n_t + n_xi + n_x);
    return t;
}

void copy_cores(tt_ctx* c, const tt_t* s, tt_t* t) {
    TT_REQUIRE(t->cap1 >= s->r1 && t->cap2 >= s->r2 && t->n_t == s->n_t && t->n_xi == s->n_xi && t->n_x == s->n_x,
               "copy_cores: destination (capacity %d, %d) cannot hold ranks (%d, %d)", t->cap1, t->cap2, s->r1, s->r2);
    t->r1 = s->r1;
    t->r2 = s->r2;
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    CUDA_CHECK(cudaMemcpyAsync(t->z1, s->z1, (size_t)s->n_t * s->r1 * sizeof(double), k, c->stream));
    CUDA_CHECK(cudaMemcpyAsync(t->z2, s->z2, (size_t)s->r1 * s->n_xi * s->r2 * sizeof(double), k, c->stream));
    CUDA_CHECK(cudaMemcpyAsync(t->z3, s->z3, (size_t)s->n_x * s->r2 * sizeof(double), k, c->stream));
}

TTPtr clone(tt_ctx* c, const tt_t* s, double scale) {
    TTPtr t = wrap(tt_alloc(c, s->n_t, s->n_xi, s->n_x, s->r1, s->r2));
    copy_cores(c, s, t.get());
    if (scale != 1.0) copy_mat(c, s->n_t, s->r1, colmaj(t->z1, s->n_t), colmaj(t->z1, s->n_t), scale);
    return t;
}

// ============================================================== concatenation
namespace {
struct CatTerm {
    const double* z1;
    const double* z2;
    const double* z3;
    const double* dcoef;
    double coef;
    int r1, r2, off1, off2;
};

// core1: out[(off1 + a) * n_t + t] = coef * z1[a * n_t + t]
__global__ void k_cat1(const CatTerm* __restrict__ T, int n_t, double* __restrict__ out) {
    const CatTerm q = T[blockIdx.y];
    const double cf = q.coef * (q.dcoef ? *q.dcoef : 1.0);
    const int tot = n_t * q.r1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x)
        out[(size_t)q.off1 * n_t + e] = cf * q.z1[e];
}
// core2 block diagonal: out[((off1 + a) * n_xi + s) * R2 + off2 + b] = z2[(a * n_xi + s) * r2 + b]
__global__ void k_cat2(const CatTerm* __restrict__ T, int n_xi, int R2, double* __restrict__ out) {
    const CatTerm q = T[blockIdx.y];
    const long long tot = (long long)q.r1 * n_xi * q.r2;
    for (long long e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e % q.r2);
        const long long as = e / q.r2;
        const int s = (int)(as % n_xi), a = (int)(as / n_xi);
        out[((size_t)(q.off1 + a) * n_xi + s) * R2 + q.off2 + b] = q.z2[e];
    }
}
// core3: out[j * R2 + off2 + b] = z3[j * r2 + b]
__global__ void k_cat3(const CatTerm* __restrict__ T, int n_x, int R2, double* __restrict__ out) {
    const CatTerm q = T[blockIdx.y];
    const long long tot = (long long)n_x * q.r2;
    for (long long e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e % q.r2);
        const long long j = e / q.r2;
        out[j * R2 + q.off2 + b] = q.z3[e];
    }
}
}  // namespace

TTPtr concat(tt_ctx* c, const std::vector<Summand>& terms) {
    TT_REQUIRE(!terms.empty(), "concat of nothing");
    const tt_t* f = terms[0].t;
    int R1 = 0, R2 = 0;
    std::vector<CatTerm> h(terms.size());
    for (size_t i = 0; i < terms.size(); ++i) {
        const tt_t* t = terms[i].t;
        TT_REQUIRE(t->n_t == f->n_t && t->n_xi == f->n_xi && t->n_x == f->n_x, "concat: shape mismatch");
        h[i] = CatTerm{t->z1, t->z2, t->z3, terms[i].dcoef, terms[i].coef, t->r1, t->r2, R1, R2};
        R1 += t->r1;
        R2 += t->r2;
    }
    TTPtr out = wrap(tt_alloc(c, f->n_t, f->n_xi, f->n_x, R1, R2));
    fill_zero(c, out->z2, (size_t)R1 * f->n_xi * R2);
    DBuf<CatTerm> dT(c, h.size());
    CUDA_CHECK(cudaMemcpyAsync(dT.p, h.data(), h.size() * sizeof(CatTerm), cudaMemcpyHostToDevice, c->stream));
    const int nt = (int)h.size();
    int maxr1 = 0, maxr2 = 0;
    for (auto& q : h) { maxr1 = std::max(maxr1, q.r1); maxr2 = std::max(maxr2, q.r2); }
    k_cat1<<<dim3(ceil_div((long long)f->n_t * maxr1, 256), nt), 256, 0, c->stream>>>(dT.p, f->n_t, out->z1);
    LAUNCH_CHECK(c);
    k_cat2<<<dim3(std::min(1024, ceil_div((long long)maxr1 * f->n_xi * maxr2, 256)), nt), 256, 0, c->stream>>>(
        dT.p, f->n_xi, R2, out->z2);
    LAUNCH_CHECK(c);
    k_cat3<<<dim3(std::min(2048, ceil_div((long long)f->n_x * maxr2, 256)), nt), 256, 0, c->stream>>>(
        dT.p, f->n_x, R2, out->z3);
    LAUNCH_CHECK(c);
    return out;
}

// ============================================================== truncation
namespace {
__global__ void k_sqrt_abs(int n, double* __restrict__ v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = sqrt(fabs(v[i]));
}
// column j (rows 0..m-1, leading dimension ld) of X scaled by sqrt(s[j]) (mode 0), by
// 1 / s[j] (mode 1; a zero s[j] gives a zero column) or by s[j] (mode 2); one block
// per column
__global__ void k_scale_cols(int m, double* __restrict__ X, int ld, const double* __restrict__ s, int mode) {
    const int j = blockIdx.x;
    const double v = s[j];
    const double f = mode == 0 ? sqrt(fabs(v)) : mode == 1 ? (v > 0.0 ? 1.0 / v : 0.0) : v;
    for (int i = threadIdx.x; i < m; i += blockDim.x) X[(size_t)j * ld + i] *= f;
}

// H = (3 I - G) / 2 in place (n x n, column-major): the Newton-Schulz step for the
// polar factor, U <- U H with G = U^T U
__global__ void k_ns_shift(int n, double* __restrict__ G) {
    const long long len = (long long)n * n;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len; t += (long long)gridDim.x * blockDim.x)
        G[t] = (t % n == t / n ? 1.5 : 0.0) - 0.5 * G[t];
}
}  // namespace

// Truncation through Gram matrices, for tolerances well above sqrt(machine eps):
// the singular values and left singular vectors of both unfoldings are the
// eigenpairs of S1 = Z(1) Z(1)^T (n_t x n_t) and, after projecting mode 1, of
// S2 = Z(2) Z(2)^T ((r1 n_xi) x (r1 n_xi)), assembled from the cores by FP64 GEMMs
// (no QR).  One-sided Jacobi on a symmetric PSD matrix returns its eigenvectors
// with column norms equal to the eigenvalues.  Eigenvalues carry an absolute
// error of order n eps_mach ||z||^2, far below delta^2 = eps^2 ||z||^2 / 2 here.
static TTPtr round_gram(tt_ctx* c, const tt_t* z, double eps, RoundOut* info, int cap1, int cap2) {
    PrecScope fp64(c, 0);
    const int n_t = z->n_t, n_xi = z->n_xi, n_x = z->n_x, R1 = z->r1, R2 = z->r2;
    // G3 = z3^T z3 costs 2 R2^2 (n_x + R1 n_xi) flops, X = z2_left z3^T costs 2 R1 n_xi R2 n_x
    const bool wide = (double)R2 * (n_x + (double)R1 * n_xi) >= (double)R1 * n_xi * n_x;
    // W2 = sum_s (z2_s F^T)(z2_s F^T)^T with F^T F = z3 z3^T-metric:
    //   narrow: G3 = z3^T z3 (R2 x R2), T = z2_left G3, W2 = z2_r T_r^T
    //   wide:   X = z2_left z3^T ((R1 n_xi) x n_x), W2 = X_r X_r^T
    DBuf<double> G3, X, W2(c, (size_t)R1 * R1);
    if (!wide) {
        G3.alloc(c, (size_t)R2 * R2);
        gemm(c, R2, R2, n_x, 1.0, trans(rowmaj(z->z3, R2)), rowmaj(z->z3, R2), 0.0, rowmaj(G3.p, R2));
        DBuf<double> T(c, (size_t)R1 * n_xi * R2);
        gemm(c, R1 * n_xi, R2, R2, 1.0, rowmaj(z->z2, R2), rowmaj(G3.p, R2), 0.0, rowmaj(T.p, R2));
        gemm(c, R1, R1, n_xi * R2, 1.0, rowmaj(z->z2, (long long)n_xi * R2), trans(rowmaj(T.p, (long long)n_xi * R2)),
             0.0, rowmaj(W2.p, R1));
    } else {
        X.alloc(c, (size_t)R1 * n_xi * n_x);
        gemm(c, R1 * n_xi, n_x, R2, 1.0, rowmaj(z->z2, R2), trans(rowmaj(z->z3, R2)), 0.0, rowmaj(X.p, n_x));
        gemm(c, R1, R1, n_xi * n_x, 1.0, rowmaj(X.p, (long long)n_xi * n_x), trans(rowmaj(X.p, (long long)n_xi * n_x)),
             0.0, rowmaj(W2.p, R1));
    }
    // S1 = z1 W2 z1^T
    DBuf<double> tmp(c, (size_t)n_t * R1), S1(c, (size_t)n_t * n_t);
    gemm(c, n_t, R1, R1, 1.0, colmaj(z->z1, n_t), rowmaj(W2.p, R1), 0.0, colmaj(tmp.p, n_t));
    gemm(c, n_t, n_t, R1, 1.0, colmaj(tmp.p, n_t), trans(colmaj(z->z1, n_t)), 0.0, colmaj(S1.p, n_t));
    DBuf<double> sig1(c, n_t), U1(c, (size_t)n_t * n_t);
    left_svd(c, n_t, n_t, colmaj(S1.p, n_t), sig1.p, U1.p);
    k_sqrt_abs<<<ceil_div(n_t, 256), 256, 0, c->stream>>>(n_t, sig1.p);
    LAUNCH_CHECK(c);
    DBuf<TruncInfo> dinfo(c, 1);
    trunc_first(c, sig1.p, n_t, eps, dinfo.p, cap1);
    TruncInfo h;
    read_back(c, dinfo.p, &h, 1);
    check_status(c);
    if (!(h.nrm == h.nrm) || std::isinf(h.nrm)) TT_THROW(TT_ENAN, "non-finite norm in truncation");
    if (h.nrm == 0.0) {
        if (info) { info->nrm_before = 0.0; info->nrm_after = 0.0; }
        return zeros(c, n_t, n_xi, n_x);
    }
    const int r1 = h.r1;
    DBuf<double> P1(c, (size_t)r1 * R1);
    gemm(c, r1, R1, n_t, 1.0, trans(colmaj(U1.p, n_t)), colmaj(z->z1, n_t), 0.0, rowmaj(P1.p, R1));
    DBuf<double> C2(c, (size_t)r1 * n_xi * R2);
    gemm(c, r1, n_xi * R2, R1, 1.0, rowmaj(P1.p, R1), rowmaj(z->z2, (long long)n_xi * R2), 0.0,
         rowmaj(C2.p, (long long)n_xi * R2));
    const int m = r1 * n_xi;
    // Left singular pairs of the second unfolding Y = C2_left z3^T (m x n_x) from the
    // smaller of two Gram matrices: S2 = Y Y^T (m x m), or, on the narrow route when
    // 2 R2^3 < m^3, B^T B (R2 x R2) with B = C2_left F and G3 = F F^T (F = eigenvectors
    // of G3 scaled by the square roots of its eigenvalues): Y Y^T = B B^T, so the
    // eigenpairs (V, Sigma^2) of B^T B give the left singular vectors U2 = B V Sigma^-1.
    const bool rside = !wide && 2.0 * R2 * R2 * (double)R2 < (double)m * m * m;
    const int p2 = rside ? R2 : m;
    DBuf<double> sig2(c, p2), U2(c, (size_t)m * p2), Bm, V;
    if (rside) {
        // F from the eigenpairs of G3 (already at hand): the same squared spectrum as
        // S2's, with no QR of the n_x-row core
        DBuf<double> lg(c, R2), Ug(c, (size_t)R2 * R2);
        left_svd(c, R2, R2, colmaj(G3.p, R2), lg.p, Ug.p);
        k_scale_cols<<<R2, 128, 0, c->stream>>>(R2, Ug.p, R2, lg.p, 0);
        LAUNCH_CHECK(c);
        Bm.alloc(c, (size_t)m * R2);
        gemm(c, m, R2, R2, 1.0, rowmaj(C2.p, R2), colmaj(Ug.p, R2), 0.0, rowmaj(Bm.p, R2));
        DBuf<double> K(c, (size_t)R2 * R2);
        gemm(c, R2, R2, m, 1.0, trans(rowmaj(Bm.p, R2)), rowmaj(Bm.p, R2), 0.0, colmaj(K.p, R2));
        V.alloc(c, (size_t)R2 * R2);
        left_svd(c, R2, R2, colmaj(K.p, R2), sig2.p, V.p);
    } else {
        DBuf<double> S2(c, (size_t)m * m);
        if (!wide) {
            DBuf<double> T2(c, (size_t)m * R2);
            gemm(c, m, R2, R2, 1.0, rowmaj(C2.p, R2), rowmaj(G3.p, R2), 0.0, rowmaj(T2.p, R2));
            gemm(c, m, m, R2, 1.0, rowmaj(T2.p, R2), trans(rowmaj(C2.p, R2)), 0.0, colmaj(S2.p, m));
        } else {
            DBuf<double> Y(c, (size_t)m * n_x);
            gemm(c, m, n_x, R2, 1.0, rowmaj(C2.p, R2), trans(rowmaj(z->z3, R2)), 0.0, rowmaj(Y.p, n_x));
            gemm(c, m, m, n_x, 1.0, rowmaj(Y.p, n_x), trans(rowmaj(Y.p, n_x)), 0.0, colmaj(S2.p, m));
        }
        left_svd(c, m, m, colmaj(S2.p, m), sig2.p, U2.p);
    }
    k_sqrt_abs<<<ceil_div(p2, 256), 256, 0, c->stream>>>(p2, sig2.p);
    LAUNCH_CHECK(c);
    trunc_second(c, sig2.p, p2, eps, dinfo.p, cap2);
    read_back(c, dinfo.p, &h, 1);
    check_status(c);
    const int r2 = h.r2;
    if (rside) {
        gemm(c, m, r2, R2, 1.0, rowmaj(Bm.p, R2), colmaj(V.p, R2), 0.0, colmaj(U2.p, m));
        k_scale_cols<<<r2, 128, 0, c->stream>>>(m, U2.p, m, sig2.p, 1);
        LAUNCH_CHECK(c);
        // U2 = B V Sigma^-1 carries V's angular error (the Jacobi tolerance) amplified by
        // sigma_max / sigma_i: its span is right to that tolerance, the orthogonality of
        // its columns is not.  Two Newton-Schulz steps U2 <- U2 (3 I - U2^T U2) / 2 take
        // it to the nearest orthonormal frame (the polar factor), same span.
        DBuf<double> G(c, (size_t)r2 * r2), U2n(c, (size_t)m * r2);
        for (int it = 0; it < 2; ++it) {
            gemm(c, r2, r2, m, 1.0, trans(colmaj(U2.p, m)), colmaj(U2.p, m), 0.0, colmaj(G.p, r2));
            k_ns_shift<<<ceil_div(r2 * r2, 256), 256, 0, c->stream>>>(r2, G.p);
            LAUNCH_CHECK(c);
            gemm(c, m, r2, r2, 1.0, colmaj(U2.p, m), colmaj(G.p, r2), 0.0, colmaj(U2n.p, m));
            CUDA_CHECK(cudaMemcpyAsync(U2.p, U2n.p, (size_t)m * r2 * sizeof(double), cudaMemcpyDeviceToDevice,
                                       c->stream));
        }
    }
    TTPtr out = wrap(tt_alloc(c, n_t, n_xi, n_x, r1, r2));
    CUDA_CHECK(cudaMemcpyAsync(out->z1, U1.p, (size_t)n_t * r1 * sizeof(double), cudaMemcpyDeviceToDevice,
                               c->stream));
    copy_mat(c, m, r2, colmaj(U2.p, m), rowmaj(out->z2, r2));
    DBuf<double> P2(c, (size_t)r2 * R2);
    gemm(c, r2, R2, m, 1.0, trans(colmaj(U2.p, m)), rowmaj(C2.p, R2), 0.0, rowmaj(P2.p, R2));
    gemm(c, n_x, r2, R2, 1.0, rowmaj(z->z3, R2), trans(rowmaj(P2.p, R2)), 0.0, rowmaj(out->z3, r2));
    if (info) {
        info->nrm_before = h.nrm;
        info->nrm_after = h.nrm_after;
        info->capped = h.capped;
    }
    static const bool log = getenv("TT_LOG_ROUND") != nullptr;
    if (log)
        fprintf(stderr, "round-gram n=(%d,%d,%d) R=(%d,%d) -> (%d,%d) eps=%.1e\n", n_t, n_xi, n_x, R1, R2, r1, r2,
                eps);
    return out;
}

// When the first rank exceeds n_t, replace z1 by an orthonormal basis U0 of its
// column space (left singular vectors, FP64) and absorb U0^T z1 into the middle
// core: the same tensor with first rank <= n_t, so every later product and factor
// of the truncation works on n_t instead of R1 rows of the middle core.
TTPtr round_tt(tt_ctx* c, const tt_t* z, double eps, RoundOut* info, int cap1, int cap2) {
    if (z->r1 > z->n_t) {
        const int n_t = z->n_t, n_xi = z->n_xi, R1 = z->r1, R2 = z->r2;
        DBuf<double> sig(c, n_t), U0(c, (size_t)n_t * n_t);
        {
            PrecScope fp64(c, 0);
            left_svd(c, n_t, R1, colmaj(z->z1, n_t), sig.p, U0.p);
        }
        DBuf<double> F1(c, (size_t)n_t * R1), z2c(c, (size_t)n_t * n_xi * R2);
        gemm(c, n_t, R1, n_t, 1.0, trans(colmaj(U0.p, n_t)), colmaj(z->z1, n_t), 0.0, rowmaj(F1.p, R1));
        gemm(c, n_t, n_xi * R2, R1, 1.0, rowmaj(F1.p, R1), rowmaj(z->z2, (long long)n_xi * R2), 0.0,
             rowmaj(z2c.p, (long long)n_xi * R2));
        tt_t view = *z;     // non-owning view: compressed cores 1, 2 and the original core 3
        view.base = nullptr;
        view.r1 = n_t;
        view.z1 = U0.p;
        view.z2 = z2c.p;
        return round_tt(c, &view, eps, info, cap1, cap2);
    }
    // plain FP64 path: Gram route for tolerances well above sqrt(eps_mach); the mixed
    // path keeps the R-factor route, whose products it runs in FP32
    if (eps >= kGramMinEps && c->gram_ok && !c->fast) return round_gram(c, z, eps, info, cap1, cap2);
    const int n_t = z->n_t, n_xi = z->n_xi, n_x = z->n_x, R1 = z->r1, R2 = z->r2;
    // 1. R3 with z3 = Q3 R3 (z3: n_x x R2 row-major, Q3 orthonormal columns).  Q3 = I
    //    with R3 = z3 is always a valid choice; a Householder R factor (k = R2 rows)
    //    pays off only when R2 is well below n_x and n_x is large: its R2 columns are
    //    sequential (one cluster barrier each), while skipping it only makes the later
    //    products and the R factors of the other unfoldings taller (measured on n_x =
    //    1312: the small solve 4% faster in mixed precision, 10% in FP64 without it).
    const bool use_qr = 4 * R2 < n_x && n_x > 4096;
    const int k = use_qr ? R2 : n_x;
    DBuf<double> R3buf;
    const double* R3 = z->z3;
    if (use_qr) {
        R3buf.alloc(c, (size_t)k * R2);
        qr_r(c, n_x, R2, rowmaj(z->z3, R2), R3buf.p, R2);
        R3 = R3buf.p;
    }
    // 2. Y2 = z2 x3 R3 : (R1 n_xi x R2) (R2 x k)
    DBuf<double> Y2(c, (size_t)R1 * n_xi * k);
    gemm(c, R1 * n_xi, k, R2, 1.0, rowmaj(z->z2, R2), trans(rowmaj(R3, R2)), 0.0, rowmaj(Y2.p, k));
    // 3. Rf2 with M2 = Q2 Rf2, M2 = (right unfolding of Y2)^T, an (n_xi k) x R1 matrix;
    //    again M2 itself when R1 >= n_xi k.  Rf2 is k1 x R1, read through (s0, s1).
    const int k1 = std::min(n_xi * k, R1);
    DBuf<double> Rf2buf;
    MatView Rf2{Y2.p, 1, (long long)n_xi * k};
    if (R1 < n_xi * k) {
        Rf2buf.alloc(c, (size_t)k1 * R1);
        qr_r(c, n_xi * k, R1, MatView{Y2.p, 1, (long long)n_xi * k}, Rf2buf.p, R1);
        Rf2 = rowmaj((const double*)Rf2buf.p, R1);
    }
    // 4. A1 = z1 Rf2^T (n_t x k1): same singular values / left vectors as the first unfolding
    DBuf<double> A1(c, (size_t)n_t * k1);
    gemm(c, n_t, k1, R1, 1.0, colmaj(z->z1, n_t), trans(Rf2), 0.0, colmaj(A1.p, n_t));
    // 5. left SVD, ||z||, delta, r1
    const int p1 = std::min(n_t, k1);
    DBuf<double> sig1(c, p1), U1(c, (size_t)n_t * p1);
    // Jacobi target matched to the truncation: columns orthogonal to 1e-3 eps leave
    // singular-value errors of order 1e-3 eps sigma_max, far from the cut at eps ||z||
    const double jtol = eps > 0.0 ? std::min(1e-8, std::max(1e-13, 1e-3 * eps)) : 1e-13;
    left_svd(c, n_t, k1, colmaj(A1.p, n_t), sig1.p, U1.p, jtol);
    DBuf<TruncInfo> dinfo(c, 1);
    trunc_first(c, sig1.p, p1, eps, dinfo.p, cap1);
    TruncInfo h;
    read_back(c, dinfo.p, &h, 1);
    check_status(c);
    if (!(h.nrm == h.nrm) || std::isinf(h.nrm)) TT_THROW(TT_ENAN, "non-finite norm in truncation");
    if (h.nrm == 0.0) {
        if (info) { info->nrm_before = 0.0; info->nrm_after = 0.0; }
        return zeros(c, n_t, n_xi, n_x);
    }
    const int r1 = h.r1;
    // 6. P1 = U1_r^T z1 (r1 x R1)
    DBuf<double> P1(c, (size_t)r1 * R1);
    gemm(c, r1, R1, n_t, 1.0, trans(colmaj(U1.p, n_t)), colmaj(z->z1, n_t), 0.0, rowmaj(P1.p, R1));
    // 7. C2 = P1 x1 z2 : [r1][n_xi][R2]
    DBuf<double> C2(c, (size_t)r1 * n_xi * R2);
    gemm(c, r1, n_xi * R2, R1, 1.0, rowmaj(P1.p, R1), rowmaj(z->z2, (long long)n_xi * R2), 0.0,
         rowmaj(C2.p, (long long)n_xi * R2));
    // 8. Y = C2_left R3^T (m x k), m = r1 n_xi
    const int m = r1 * n_xi;
    DBuf<double> Y(c, (size_t)m * k);
    gemm(c, m, k, R2, 1.0, rowmaj(C2.p, R2), trans(rowmaj(R3, R2)), 0.0, colmaj(Y.p, m));
    // 9. left SVD of Y, r2
    const int p2 = std::min(m, k);
    DBuf<double> sig2(c, p2), U2(c, (size_t)m * p2);
    left_svd(c, m, k, colmaj(Y.p, m), sig2.p, U2.p, jtol);
    trunc_second(c, sig2.p, p2, eps, dinfo.p, cap2);
    read_back(c, dinfo.p, &h, 1);
    check_status(c);
    const int r2 = h.r2;
    TTPtr out = wrap(tt_alloc(c, n_t, n_xi, n_x, r1, r2));
    // 10. new cores 1 and 2 are the kept left singular frames
    CUDA_CHECK(cudaMemcpyAsync(out->z1, U1.p, (size_t)n_t * r1 * sizeof(double), cudaMemcpyDeviceToDevice,
                               c->stream));
    copy_mat(c, m, r2, colmaj(U2.p, m), rowmaj(out->z2, r2));
    // 11-12. new z3 = z3 P2^T with P2 = U2_r^T C2_left (r2 x R2)
    DBuf<double> P2(c, (size_t)r2 * R2);
    gemm(c, r2, R2, m, 1.0, trans(colmaj(U2.p, m)), rowmaj(C2.p, R2), 0.0, rowmaj(P2.p, R2));
    gemm(c, n_x, r2, R2, 1.0, rowmaj(z->z3, R2), trans(rowmaj(P2.p, R2)), 0.0, rowmaj(out->z3, r2));
    if (info) {
        info->nrm_before = h.nrm;
        info->nrm_after = h.nrm_after;
        info->capped = h.capped;
    }
    static const bool log = getenv("TT_LOG_ROUND") != nullptr;
    if (log)
        fprintf(stderr, "round n=(%d,%d,%d) R=(%d,%d) -> (%d,%d) eps=%.1e fast=%d\n", n_t, n_xi, n_x, R1, R2, r1,
                r2, eps, c->fast);
    return out;
}

// T_eps of a velocity train and a pressure train at once: the pressure train is
// truncated on the side context's stream from a second host thread while the
// velocity train is truncated on the context's own stream (the two truncations
// share no data; each synchronises its own stream for its ranks).  The results are
// those of two consecutive round_tt calls; the pressure result is handed back to the
// context (its memory is released in the context's stream order).
TTPtr round_any(tt_ctx* c, const tt_t* z, double eps, RoundOut* info) {
    if (!c->randomized) return round_tt(c, z, eps, info);
    const unsigned long long seed = c->rand_seq;
    c->rand_seq = c->rand_seq * 6364136223846793005ull + 1442695040888963407ull;
    return round_rand(c, z, eps, seed, info);
}

void round_pair(tt_ctx* c, const tt_t* u, const tt_t* p, double eps, TTPtr* ru, TTPtr* rp, RoundOut* iu,
                RoundOut* ip) {
    tt_ctx* s = side_ctx(c);
    s->fast = c->fast;
    s->randomized = c->randomized;
    s->rand_seq = c->rand_seq ^ 0x9E3779B97F4A7C15ull;
    c->rand_seq = c->rand_seq * 6364136223846793005ull + 1442695040888963407ull;
    s->alloc_fn = c->alloc_fn;
    s->free_fn = c->free_fn;
    s->alloc_user = c->alloc_user;
    CUDA_CHECK(cudaEventRecord(c->ev_fork, c->stream));
    CUDA_CHECK(cudaStreamWaitEvent(s->stream, c->ev_fork, 0));
    TTPtr outp{nullptr, tt_free};
    std::exception_ptr perr;
    std::thread th([&]() {
        try {
            CUDA_CHECK(cudaSetDevice(s->device));
            outp = round_any(s, p, eps, ip);
        } catch (...) {
            perr = std::current_exception();
        }
    });
    std::exception_ptr uerr;
    try {
        *ru = round_any(c, u, eps, iu);
    } catch (...) {
        uerr = std::current_exception();
    }
    th.join();
    c->launches += s->launches;
    s->launches = 0;
    CUDA_CHECK(cudaEventRecord(c->ev_join, s->stream));
    CUDA_CHECK(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    if (uerr) std::rethrow_exception(uerr);
    if (perr) std::rethrow_exception(perr);
    outp->ctx = c;
    *rp = std::move(outp);
}

// ============================================================== inner products
namespace {
__global__ void k_frob_dot(int n, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(a[i], b[i], s);
    __shared__ double red[32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0) *out = s;
    }
}
}  // namespace

void dot_dev(tt_ctx* c, const tt_t* a, const tt_t* b, double* dout) {
    TT_REQUIRE(a->n_t == b->n_t && a->n_xi == b->n_xi && a->n_x == b->n_x, "dot: shape mismatch");
    PrecScope fp64(c, 0);   // inner products of the Arnoldi process stay FP64
    const int n_t = a->n_t, n_xi = a->n_xi, n_x = a->n_x;
    const int ra1 = a->r1, ra2 = a->r2, rb1 = b->r1, rb2 = b->r2;
    DBuf<double> W1(c, (size_t)ra1 * rb1);
    gemm(c, ra1, rb1, n_t, 1.0, trans(colmaj(a->z1, n_t)), colmaj(b->z1, n_t), 0.0, rowmaj(W1.p, rb1));
    DBuf<double> T(c, (size_t)ra1 * n_xi * rb2);
    gemm(c, ra1, n_xi * rb2, rb1, 1.0, rowmaj(W1.p, rb1), rowmaj(b->z2, (long long)n_xi * rb2), 0.0,
         rowmaj(T.p, (long long)n_xi * rb2));
    DBuf<double> W2(c, (size_t)ra2 * rb2);
    gemm(c, ra2, rb2, ra1 * n_xi, 1.0, trans(rowmaj(a->z2, ra2)), rowmaj(T.p, rb2), 0.0, rowmaj(W2.p, rb2));
    DBuf<double> G3(c, (size_t)ra2 * rb2);
    gemm(c, ra2, rb2, n_x, 1.0, trans(rowmaj(a->z3, ra2)), rowmaj(b->z3, rb2), 0.0, rowmaj(G3.p, rb2));
    k_frob_dot<<<1, 256, 0, c->stream>>>(ra2 * rb2, W2.p, G3.p, dout);
    LAUNCH_CHECK(c);
}

double dot_host(tt_ctx* c, const tt_t* a, const tt_t* b) {
    DBuf<double> d(c, 1);
    dot_dev(c, a, b, d.p);
    double h;
    read_back(c, d.p, &h, 1);
    return h;
}

}  // namespace tt
