// Randomized truncation (an opt-in variant of T_eps, Section 4.1): a Gaussian sketch of
// the row space of the second unfolding replaces the last core, whose rank R2 after a
// matvec or a Krylov sum is often many times the rank that survives, by an orthonormal
// basis of ell columns; the deterministic T_eps then runs on the small train.  The
// energy the sketch misses is estimated with independent Gaussian probes and the
// sketch widens (ell doubles) until ten times that estimate is at most a tenth of the
// truncation budget; the small train is truncated with the rest of the budget, so
// ||T(z) - z|| <= eps ||z|| holds with high probability; the deterministic
// route is used when the sketch would not be narrower than R2.  Randomized low-rank
// approximation with a posteriori probe estimates in the sense of Halko, Martinsson and
// Tropp (SIAM Review 2011); for TT rounding cf. Al Daas, Ballard et al. (SISC 2023).
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "tt.cuh"

namespace tt {
namespace {

// SplitMix64 (Steele, Lea and Flood 2014) on the counter `seed + i`, two draws turned
// into one standard normal by the Box-Muller transform.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
__global__ void k_gauss(long long n, uint64_t seed, double* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const uint64_t a = splitmix64(seed + 2 * (uint64_t)i), b = splitmix64(seed + 2 * (uint64_t)i + 1);
        const double u1 = ((double)(a >> 11) + 1.0) * 0x1.0p-53;   // (0, 1]
        const double u2 = (double)(b >> 11) * 0x1.0p-53;            // [0, 1)
        out[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
}

// Q[(a s), j] = P[a, j] O2[s, j]: the Khatri-Rao test matrix of the first two modes
// contracted with z1 (P = z1^T O1, R1 x ell row-major; O2 n_xi x ell row-major).
__global__ void k_khatri_rao(int R1, int n_xi, int ell, const double* __restrict__ P, const double* __restrict__ O2,
                             double* __restrict__ Q) {
    const long long tot = (long long)R1 * n_xi * ell;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e % ell);
        const long long as = e / ell;
        const int s = (int)(as % n_xi), a = (int)(as / n_xi);
        Q[e] = P[(size_t)a * ell + j] * O2[(size_t)s * ell + j];
    }
}

// column j of X (rows m, leading dimension ld) times 1/sqrt(lam[j]) if lam[j] > thr
// (thr = rel * lam[0], lam descending), else zero
__global__ void k_inv_sqrt_cols(int m, double* __restrict__ X, int ld, const double* __restrict__ lam, double rel) {
    const int j = blockIdx.x;
    const double l = lam[j], thr = rel * lam[0];
    const double f = (l > thr && l > 0.0) ? 1.0 / sqrt(l) : 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) X[(size_t)j * ld + i] *= f;
}

__global__ void k_sumsq(long long n, const double* __restrict__ x, double* __restrict__ out) {
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s = fma(x[i], x[i], s);
    __shared__ double red[32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0) atomicAdd(out, s);
    }
}

void gauss(tt_ctx* c, long long n, uint64_t seed, double* out) {
    k_gauss<<<(int)std::min<long long>(1024, (n + 255) / 256), 256, 0, c->stream>>>(n, seed, out);
    LAUNCH_CHECK(c);
}

// B (n x k, column-major, ld n) := an orthonormal basis of range(Y) (Y n x ell, column-major),
// from the eigenpairs of Y^T Y: directions with eigenvalue below 1e-14 of the largest are
// dropped (their energy is far below any truncation threshold); a second pass on B^T B
// restores the orthogonality the first loses to rounding.  Returns k.
int orth_basis(tt_ctx* c, int n, int ell, const double* Y, DBuf<double>& B) {
    DBuf<double> cur(c, (size_t)n * ell);
    CUDA_CHECK(cudaMemcpyAsync(cur.p, Y, (size_t)n * ell * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    for (int pass = 0; pass < 2; ++pass) {
        DBuf<double> G(c, (size_t)ell * ell), lam(c, ell), V(c, (size_t)ell * ell);
        gemm(c, ell, ell, n, 1.0, trans(colmaj(cur.p, n)), colmaj(cur.p, n), 0.0, colmaj(G.p, ell));
        left_svd(c, ell, ell, colmaj(G.p, ell), lam.p, V.p);
        k_inv_sqrt_cols<<<ell, 128, 0, c->stream>>>(ell, V.p, ell, lam.p, 1e-14);
        LAUNCH_CHECK(c);
        DBuf<double> nxt(c, (size_t)n * ell);
        gemm(c, n, ell, ell, 1.0, colmaj(cur.p, n), colmaj(V.p, ell), 0.0, colmaj(nxt.p, n));
        cur = std::move(nxt);
    }
    B = std::move(cur);
    return ell;
}
}  // namespace

TTPtr round_rand(tt_ctx* c, const tt_t* z, double eps, uint64_t seed, RoundOut* info, int* ell_used) {
    const int n_t = z->n_t, n_xi = z->n_xi, n_x = z->n_x, R1 = z->r1, R2 = z->r2;
    if (ell_used) *ell_used = R2;
    if (eps <= 0.0 || R2 <= kRandMinRank) return round_tt(c, z, eps, info);
    constexpr int q = 8;   // probes of the discarded energy
    int ell = std::max(kRandMinRank / 2, (R2 + 3) / 4);
    for (int attempt = 0; ell < R2 && ell < n_x; ++attempt, ell = std::min(R2, 2 * ell)) {
        const uint64_t sd = seed * 0x2545F4914F6CDD1Dull + (uint64_t)(attempt + 1) * 0x9E3779B97F4A7C15ull;
        // sketch of the row space of X(2) ((n_t n_xi) x n_x): Y = X(2)^T (O1 (.) O2) =
        // z3 z2_left^T Q, Q[(a s), j] = (z1^T O1)[a, j] O2[s, j]
        DBuf<double> O1(c, (size_t)n_t * ell), O2(c, (size_t)n_xi * ell), P(c, (size_t)R1 * ell);
        gauss(c, (long long)n_t * ell, sd, O1.p);
        gauss(c, (long long)n_xi * ell, sd ^ 0x5851F42D4C957F2Dull, O2.p);
        gemm(c, R1, ell, n_t, 1.0, trans(colmaj(z->z1, n_t)), rowmaj(O1.p, ell), 0.0, rowmaj(P.p, ell));
        DBuf<double> Q(c, (size_t)R1 * n_xi * ell);
        k_khatri_rao<<<(int)std::min<long long>(4096, ((long long)R1 * n_xi * ell + 255) / 256), 256, 0, c->stream>>>(
            R1, n_xi, ell, P.p, O2.p, Q.p);
        LAUNCH_CHECK(c);
        DBuf<double> W(c, (size_t)R2 * ell), Y(c, (size_t)n_x * ell);
        gemm(c, R2, ell, R1 * n_xi, 1.0, trans(rowmaj(z->z2, R2)), rowmaj(Q.p, ell), 0.0, rowmaj(W.p, ell));
        gemm(c, n_x, ell, R2, 1.0, rowmaj(z->z3, R2), rowmaj(W.p, ell), 0.0, colmaj(Y.p, n_x));
        // the basis, the probes and the compressed train in FP64 on every path: the probe
        // residuals resolve energies near eps^2 ||z||^2
        PrecScope fp64(c, 0);
        DBuf<double> B;
        orth_basis(c, n_x, ell, Y.p, B);
        // probes y_i = X(2)^T g_i, g_i (n_t x n_xi) Gaussian: y_i = z3 z2_left^T vec(z1^T g_i)
        DBuf<double> Gp(c, (size_t)q * n_t * n_xi), Hv(c, (size_t)R1 * n_xi * q);
        gauss(c, (long long)q * n_t * n_xi, sd ^ 0xD1B54A32D192ED03ull, Gp.p);
        for (int i = 0; i < q; ++i)
            gemm(c, R1, n_xi, n_t, 1.0, trans(colmaj(z->z1, n_t)), rowmaj(Gp.p + (size_t)i * n_t * n_xi, n_xi), 0.0,
                 MatViewMut{Hv.p + i, (long long)n_xi * q, q});
        DBuf<double> Wp(c, (size_t)R2 * q), Yp(c, (size_t)n_x * q), Cp(c, (size_t)ell * q);
        gemm(c, R2, q, R1 * n_xi, 1.0, trans(rowmaj(z->z2, R2)), rowmaj(Hv.p, q), 0.0, rowmaj(Wp.p, q));
        gemm(c, n_x, q, R2, 1.0, rowmaj(z->z3, R2), rowmaj(Wp.p, q), 0.0, colmaj(Yp.p, n_x));
        gemm(c, ell, q, n_x, 1.0, trans(colmaj(B.p, n_x)), colmaj(Yp.p, n_x), 0.0, colmaj(Cp.p, ell));
        gemm(c, n_x, q, ell, -1.0, colmaj(B.p, n_x), colmaj(Cp.p, ell), 1.0, colmaj(Yp.p, n_x));
        DBuf<double> e2d(c, 1);
        CUDA_CHECK(cudaMemsetAsync(e2d.p, 0, sizeof(double), c->stream));
        k_sumsq<<<64, 256, 0, c->stream>>>((long long)n_x * q, Yp.p, e2d.p);
        LAUNCH_CHECK(c);
        // the compressed train: cores z1, z2_left (z3^T B), B
        TTPtr xt = wrap(tt_alloc(c, n_t, n_xi, n_x, R1, ell));
        CUDA_CHECK(cudaMemcpyAsync(xt->z1, z->z1, (size_t)n_t * R1 * sizeof(double), cudaMemcpyDeviceToDevice,
                                   c->stream));
        DBuf<double> M(c, (size_t)R2 * ell);
        gemm(c, R2, ell, n_x, 1.0, trans(rowmaj(z->z3, R2)), colmaj(B.p, n_x), 0.0, rowmaj(M.p, ell));
        gemm(c, R1 * n_xi, ell, R2, 1.0, rowmaj(z->z2, R2), rowmaj(M.p, ell), 0.0, rowmaj(xt->z2, ell));
        copy_mat(c, n_x, ell, colmaj(B.p, n_x), rowmaj(xt->z3, ell));
        double e2 = 0.0;
        read_back(c, (const double*)e2d.p, &e2, 1);
        e2 /= q;
        const double nt2 = dot_host(c, xt.get(), xt.get());
        if (!(nt2 == nt2) || std::isinf(nt2) || !(e2 == e2)) TT_THROW(TT_ENAN, "non-finite norm in truncation");
        // accept when ten times the estimated missed energy is at most 10% of the budget;
        // the small train is then truncated with what remains (at least 90%)
        if (10.0 * e2 <= 0.1 * eps * eps * (nt2 + e2) || nt2 == 0.0) {
            const double tot2 = nt2 + e2;
            const double eps2 = std::max(eps * eps * tot2 - 10.0 * e2, 0.5 * eps * eps * tot2) / std::max(nt2, 1e-300);
            RoundOut ri;
            TTPtr out = round_tt(c, xt.get(), std::sqrt(eps2), &ri);
            if (info) {
                info->nrm_before = std::sqrt(tot2);
                info->nrm_after = ri.nrm_after;
                info->capped = ri.capped;
            }
            if (ell_used) *ell_used = ell;
            return out;
        }
    }
    return round_tt(c, z, eps, info);
}

}  // namespace tt
