// Dense FP64 building blocks of the TT rounding (Section 4.1): strided GEMM,
// R factor of a tall matrix by Householder reflections, left singular vectors
// by one-sided Jacobi.
#pragma once
#include "common.cuh"

namespace tt {

// Strided matrix view: element (i, j) at p[i * s0 + j * s1].
struct MatView {
    const double* p;
    long long s0, s1;
};
struct MatViewMut {
    double* p;
    long long s0, s1;
    operator MatView() const { return MatView{p, s0, s1}; }
};
inline MatView rowmaj(const double* p, long long ld) { return {p, ld, 1}; }
inline MatView colmaj(const double* p, long long ld) { return {p, 1, ld}; }
inline MatView trans(MatView v) { return {v.p, v.s1, v.s0}; }
inline MatViewMut rowmaj(double* p, long long ld) { return {p, ld, 1}; }
inline MatViewMut colmaj(double* p, long long ld) { return {p, 1, ld}; }

// C (M x N) = alpha A (M x K) B (K x N) + beta C.  beta == 0 never reads C.
void gemm(tt_ctx* c, int M, int N, int K, double alpha, MatView A, MatView B, double beta,
          MatViewMut C);
// Same, with split-K partial sums in a caller workspace of ws_len doubles (no
// allocation; split-K shrinks to what fits, down to none).
void gemm_ws(tt_ctx* c, int M, int N, int K, double alpha, MatView A, MatView B, double beta,
             MatViewMut C, double* ws, size_t ws_len);

// R factor (k x c upper trapezoidal, k = min(n, c), row-major with leading
// dimension ldr) of the n x c matrix A by Householder QR.  Q is not formed.
void qr_r(tt_ctx* c, int n, int cols, MatView A, double* R, int ldr);

// Left singular vectors and singular values of the m x n matrix A (any strides).
// Writes sig (p = min(m, n) values, descending) and U (m x p, column-major,
// ld m; column i belongs to sig[i]; columns of zero singular values are zero).
// ortho_tol: Jacobi stops when every column pair has |a.b| <= ortho_tol |a||b|
// (at least 4 m eps_mach); singular values then carry absolute errors of order
// ortho_tol * sigma_max.
void left_svd(tt_ctx* c, int m, int n, MatView A, double* sig, double* U, double ortho_tol = 1e-13);

// Truncation of Section 4.1 on device data: given sorted sig1 (p1) and sig2 (p2)
// it is applied in two calls; see trunc.cu.
struct TruncInfo {
    double nrm;        // ||z||
    double delta2;     // delta^2 = (eps ||z||)^2 / 2
    double nrm_after;  // ||T(z)||
    int r1, r2;
    int capped;        // bit 0: r1 was cut to its cap, bit 1: r2 was
};
// First stage: nrm^2 = sum sig1^2, delta2, r1 (at most maxr when maxr > 0).
void trunc_first(tt_ctx* c, const double* sig1, int p1, double eps, TruncInfo* dinfo, int maxr = 0);
// Second stage: r2 (at most maxr when maxr > 0) and nrm_after from sig2.
void trunc_second(tt_ctx* c, const double* sig2, int p2, double eps, TruncInfo* dinfo, int maxr = 0);

// Copy / transpose a strided matrix into a strided destination (m x n).
void copy_mat(tt_ctx* c, int m, int n, MatView A, MatViewMut B, double alpha = 1.0);
void fill_zero(tt_ctx* c, double* p, size_t n);

}  // namespace tt
