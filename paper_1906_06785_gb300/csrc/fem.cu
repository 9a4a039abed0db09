// Discretisation on the device (Sections 3.2, 5.1): Q2-Q1 element matrices of
// eq. (mat_entries) and of B, assembled by deterministic gathers into CSR
// patterns over free (f) and Dirichlet (D) velocity dofs; gPC matrices G_l, H_l;
// sparse products with velocity / pressure trains; banded LU for the mean
// velocity matrix and the pressure Laplacian B M*^-1 B^T (Section 5.1).
//
// All elements are squares of side h; element-local matrices are integrated
// with 3 x 3 Gauss points on the unit square.  Local velocity node a + 3b sits
// at (a/2, b/2), local pressure vertex a + 2b at (a, b).
#include <algorithm>
#include <cmath>
#include <numeric>

#include "problem.cuh"

namespace tt {

// ============================================================== reference tables
__constant__ double c_phi[9][9];   // [q][i]
__constant__ double c_ds[9][9];
__constant__ double c_dt[9][9];
__constant__ double c_chi[9][4];
__constant__ double c_chs[9][4];   // d chi / ds (bilinear pressure basis)
__constant__ double c_cht[9][4];   // d chi / dt
__constant__ double c_w[9];

static void upload_tables() {
    const double g[3] = {0.5 - 0.5 * std::sqrt(0.6), 0.5, 0.5 + 0.5 * std::sqrt(0.6)};
    const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    auto L = [](int a, double s) {
        return a == 0 ? 2.0 * (s - 0.5) * (s - 1.0) : (a == 1 ? 4.0 * s * (1.0 - s) : 2.0 * s * (s - 0.5));
    };
    auto dL = [](int a, double s) { return a == 0 ? 4.0 * s - 3.0 : (a == 1 ? 4.0 - 8.0 * s : 4.0 * s - 1.0); };
    double phi[9][9], ds[9][9], dt[9][9], chi[9][4], chs[9][4], cht[9][4], w[9];
    for (int qt = 0; qt < 3; ++qt)
        for (int qs = 0; qs < 3; ++qs) {
            const int q = qs + 3 * qt;
            const double s = g[qs], t = g[qt];
            w[q] = gw[qs] * gw[qt];
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) {
                    phi[q][a + 3 * b] = L(a, s) * L(b, t);
                    ds[q][a + 3 * b] = dL(a, s) * L(b, t);
                    dt[q][a + 3 * b] = L(a, s) * dL(b, t);
                }
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    chi[q][a + 2 * b] = (a ? s : 1.0 - s) * (b ? t : 1.0 - t);
                    chs[q][a + 2 * b] = (a ? 1.0 : -1.0) * (b ? t : 1.0 - t);
                    cht[q][a + 2 * b] = (a ? s : 1.0 - s) * (b ? 1.0 : -1.0);
                }
        }
    CUDA_CHECK(cudaMemcpyToSymbol(c_phi, phi, sizeof(phi)));
    CUDA_CHECK(cudaMemcpyToSymbol(c_ds, ds, sizeof(ds)));
    CUDA_CHECK(cudaMemcpyToSymbol(c_dt, dt, sizeof(dt)));
    CUDA_CHECK(cudaMemcpyToSymbol(c_chi, chi, sizeof(chi)));
    CUDA_CHECK(cudaMemcpyToSymbol(c_chs, chs, sizeof(chs)));
    CUDA_CHECK(cudaMemcpyToSymbol(c_cht, cht, sizeof(cht)));
    CUDA_CHECK(cudaMemcpyToSymbol(c_w, w, sizeof(w)));
}

// ============================================================== element kernels
namespace {
// grid (n_elem, nf): local[f][e][i*9 + j]
__global__ void k_local_mass(int n_elem, double h, double* __restrict__ loc) {
    const int e = blockIdx.x, t = threadIdx.x;
    if (t >= 81) return;
    const int i = t / 9, j = t % 9;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) s += c_w[q] * c_phi[q][i] * c_phi[q][j];
    loc[(size_t)e * 81 + t] = s * h * h;
}

__global__ void k_local_stiff(int n_elem, int n_p, const int* __restrict__ eq1, const double* __restrict__ nu,
                              double* __restrict__ loc) {
    const int e = blockIdx.x, f = blockIdx.y, t = threadIdx.x;
    __shared__ double nuq[9];
    if (t < 9) {
        double v = 0.0;
        for (int p = 0; p < 4; ++p) v += c_chi[t][p] * nu[(size_t)f * n_p + eq1[e * 4 + p]];
        nuq[t] = v;
    }
    __syncthreads();
    if (t >= 81) return;
    const int i = t / 9, j = t % 9;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) s += c_w[q] * nuq[q] * (c_ds[q][i] * c_ds[q][j] + c_dt[q][i] * c_dt[q][j]);
    loc[((size_t)f * n_elem + e) * 81 + t] = s;
}

// w_f(node) = (W[node*ldw + f], W[(n_nodes + node)*ldw + f])
__global__ void k_local_conv(int n_elem, int n_nodes, double h, const int* __restrict__ eq2,
                             const double* __restrict__ W, int ldw, double* __restrict__ loc) {
    const int e = blockIdx.x, f = blockIdx.y, t = threadIdx.x;
    __shared__ double wn[2][9], wq[2][9];
    if (t < 18) {
        const int c = t / 9, a = t % 9;
        wn[c][a] = W[((size_t)c * n_nodes + eq2[e * 9 + a]) * ldw + f];
    }
    __syncthreads();
    if (t < 18) {
        const int c = t / 9, q = t % 9;
        double v = 0.0;
        for (int a = 0; a < 9; ++a) v += c_phi[q][a] * wn[c][a];
        wq[c][q] = v;
    }
    __syncthreads();
    if (t >= 81) return;
    const int i = t / 9, j = t % 9;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) s += c_w[q] * (wq[0][q] * c_ds[q][j] + wq[1][q] * c_dt[q][j]) * c_phi[q][i];
    loc[((size_t)f * n_elem + e) * 81 + t] = s * h;
}

// local[c][e][p*9 + j] = -h sum_q w chi_p dphi_j/d(s or t)
__global__ void k_local_div(int n_elem, double h, double* __restrict__ loc) {
    const int e = blockIdx.x, c = blockIdx.y, t = threadIdx.x;
    if (t >= 36) return;
    const int p = t / 9, j = t % 9;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) s += c_w[q] * c_chi[q][p] * (c == 0 ? c_ds[q][j] : c_dt[q][j]);
    loc[((size_t)c * n_elem + e) * 36 + t] = -s * h;
}

// Q1 pressure-space element matrices (Section 5.2, the pressure analogues of M, A_0
// and N(w) for the PCD approximation), 16 entries per element, local vertex a + 2b:
//   mass:       h^2 sum_q w chi_i chi_j
//   diffusion:  sum_q w nu_q (dchi_i/ds dchi_j/ds + dchi_i/dt dchi_j/dt)   (nu row 0: mean)
//   convection: h sum_q w (w1 dchi_j/ds + w2 dchi_j/dt) chi_i, w the Q2 field f
__global__ void k_local_pmat(int n_elem, int n_p, double h, const int* __restrict__ eq1, const double* __restrict__ nu,
                             double* __restrict__ loc) {
    const int e = blockIdx.x, kind = blockIdx.y, t = threadIdx.x;
    __shared__ double nuq[9];
    if (t < 9) {
        double v = 0.0;
        for (int p = 0; p < 4; ++p) v += c_chi[t][p] * nu[eq1[e * 4 + p]];
        nuq[t] = v;
    }
    __syncthreads();
    if (t >= 16) return;
    const int i = t / 4, j = t % 4;
    double s = 0.0;
    if (kind == 0) {
#pragma unroll
        for (int q = 0; q < 9; ++q) s += c_w[q] * c_chi[q][i] * c_chi[q][j];
        s *= h * h;
    } else {
#pragma unroll
        for (int q = 0; q < 9; ++q) s += c_w[q] * nuq[q] * (c_chs[q][i] * c_chs[q][j] + c_cht[q][i] * c_cht[q][j]);
    }
    loc[((size_t)kind * n_elem + e) * 16 + t] = s;
}

__global__ void k_local_pconv(int n_elem, int n_nodes, double h, const int* __restrict__ eq2,
                              const double* __restrict__ W, int ldw, double* __restrict__ loc) {
    const int e = blockIdx.x, f = blockIdx.y, t = threadIdx.x;
    __shared__ double wn[2][9], wq[2][9];
    if (t < 18) {
        const int c = t / 9, a = t % 9;
        wn[c][a] = W[((size_t)c * n_nodes + eq2[e * 9 + a]) * ldw + f];
    }
    __syncthreads();
    if (t < 18) {
        const int c = t / 9, q = t % 9;
        double v = 0.0;
        for (int a = 0; a < 9; ++a) v += c_phi[q][a] * wn[c][a];
        wq[c][q] = v;
    }
    __syncthreads();
    if (t >= 16) return;
    const int i = t / 4, j = t % 4;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) s += c_w[q] * (wq[0][q] * c_chs[q][j] + wq[1][q] * c_cht[q][j]) * c_chi[q][i];
    loc[((size_t)f * n_elem + e) * 16 + t] = s * h;
}

// vals[f*nnz + s] = sum_{t in gather(s)} loc[f*L + idx[t]]
__global__ void k_gather(int nnz, int nf, long long L, const int* __restrict__ ptr, const int* __restrict__ idx,
                         const double* __restrict__ loc, double* __restrict__ vals) {
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)nnz * nf) return;
    const int f = (int)(id / nnz), s = (int)(id % nnz);
    double v = 0.0;
    for (int t = ptr[s]; t < ptr[s + 1]; ++t) v += loc[(size_t)f * L + idx[t]];
    vals[(size_t)f * nnz + s] = v;
}

__global__ void k_take(int n, const int* __restrict__ perm, const double* __restrict__ src, double* __restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[perm[i]];
}

// band[i][j - i + bw] (+)= vals over the ff pattern
__global__ void k_scatter_band(int n, int bw, const int* __restrict__ rowptr, const int* __restrict__ col,
                               const double* __restrict__ vals, double* __restrict__ ab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int W = 2 * bw + 1;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) ab[(size_t)i * W + col[k] - i + bw] = vals[k];
}

// K = tau^-1 M + A_0 (+ N) on the ff pattern
__global__ void k_axpy3(int n, double a, const double* __restrict__ x, const double* __restrict__ y,
                        const double* __restrict__ z, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + y[i] + (z ? z[i] : 0.0);
}

// L_p = B M*^-1 B^T into band storage, one thread per pressure row (deterministic)
__global__ void k_lp_band(int n_p, int bw, const int* __restrict__ brp, const int* __restrict__ bcol,
                          const double* __restrict__ bx, const double* __restrict__ by,
                          const int* __restrict__ trp, const int* __restrict__ tcol, const double* __restrict__ tx,
                          const double* __restrict__ ty, const double* __restrict__ mstar, double* __restrict__ ab) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_p) return;
    const int W = 2 * bw + 1;
    for (int k = brp[p]; k < brp[p + 1]; ++k) {
        const int j = bcol[k];
        const double inv = 1.0 / mstar[j];
        for (int t = trp[j]; t < trp[j + 1]; ++t) {
            const int q = tcol[t];
            ab[(size_t)p * W + q - p + bw] += (bx[k] * tx[t] + by[k] * ty[t]) * inv;
        }
    }
}
}  // namespace

// ============================================================== sparse products
namespace {
template <typename TC>
__global__ void __launch_bounds__(256)
k_spmm_vel(VelSpmm s, const double* __restrict__ X, int ldx, double* __restrict__ Y, int ldy, int ncol) {
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wg >= s.ncomp * s.n_rows) return;
    const int comp = wg / s.n_rows, i = wg % s.n_rows;
    const double* Xc = X + (size_t)comp * s.n_in * ldx;
    double* Yr = Y + ((size_t)comp * s.n_rows + i) * ldy;
    const int k0 = s.rowptr[i], k1 = s.rowptr[i + 1];
    for (int b0 = 0; b0 < ncol; b0 += 32) {
        const int b = b0 + lane;
        const bool act = b < ncol;
        TC acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = TC(0);
        for (int k = k0; k < k1; ++k) {
            const int cl = s.col[k];
            const TC x = act ? TC(Xc[(size_t)cl * ldx + b]) : TC(0);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q < s.nmat) acc[q] = fma(TC(s.vals[q][k]), x, acc[q]);
        }
        if (act) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q < s.nmat) Yr[s.coff[q] + b] = s.coef[q] * (double)acc[q];
        }
    }
}

__global__ void k_spmm_div(int n_rows, const int* __restrict__ rp, const int* __restrict__ cl,
                           const double* __restrict__ bx, const double* __restrict__ by, int n_in, double coef,
                           const double* __restrict__ X, int ldx, double* __restrict__ Y, int ldy, int coff, int ncol) {
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wg >= n_rows) return;
    for (int b0 = 0; b0 < ncol; b0 += 32) {
        const int b = b0 + lane;
        if (b >= ncol) break;
        double acc = 0.0;
        for (int k = rp[wg]; k < rp[wg + 1]; ++k) {
            const int j = cl[k];
            acc = fma(bx[k], X[(size_t)j * ldx + b], acc);
            acc = fma(by[k], X[((size_t)n_in + j) * ldx + b], acc);
        }
        Y[(size_t)wg * ldy + coff + b] = coef * acc;
    }
}

__global__ void k_spmm_grad(int n_rows, const int* __restrict__ rp, const int* __restrict__ cl,
                            const double* __restrict__ tx, const double* __restrict__ ty, double coef,
                            const double* __restrict__ X, int ldx, double* __restrict__ Y, int ldy, int coff, int ncol) {
    const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wg >= 2 * n_rows) return;
    const int comp = wg / n_rows, j = wg % n_rows;
    const double* v = comp == 0 ? tx : ty;
    for (int b0 = 0; b0 < ncol; b0 += 32) {
        const int b = b0 + lane;
        if (b >= ncol) break;
        double acc = 0.0;
        for (int k = rp[j]; k < rp[j + 1]; ++k) acc = fma(v[k], X[(size_t)cl[k] * ldx + b], acc);
        Y[((size_t)comp * n_rows + j) * ldy + coff + b] = coef * acc;
    }
}
}  // namespace

void spmm_vel(tt_ctx* c, const VelSpmm& s, const double* X, int ldx, double* Y, int ldy, int ncol) {
    TT_REQUIRE(s.nmat >= 1 && s.nmat <= 8, "spmm_vel: nmat %d", s.nmat);
    TT_REQUIRE(s.ncomp == 1 || s.ncomp == 2, "spmm_vel: ncomp %d", s.ncomp);
    const long long threads = (long long)s.ncomp * s.n_rows * 32;
    // algorithmic bytes: pattern + nmat value arrays once, X once, Y once
    const double nnz = s.nnz;
    ProfScope prof(c, PROF_SPMM, 2.0 * s.ncomp * nnz * ncol * s.nmat,
                   (double)nnz * (4 + 8 * s.nmat) + 4.0 * (s.n_rows + 1) + 8.0 * s.ncomp * s.n_in * ncol +
                       8.0 * s.ncomp * s.n_rows * ncol * s.nmat);
    (c->fast ? k_spmm_vel<float> : k_spmm_vel<double>)<<<ceil_div(threads, 256), 256, 0, c->stream>>>(
        s, X, ldx, Y, ldy, ncol);
    LAUNCH_CHECK(c);
}
void spmm_div(tt_ctx* c, const Csr& B, const double* Bx, const double* By, int n_in, double coef,
              const double* X, int ldx, double* Y, int ldy, int coff, int ncol) {
    const long long threads = (long long)B.n_rows * 32;
    k_spmm_div<<<ceil_div(threads, 256), 256, 0, c->stream>>>(B.n_rows, B.rowptr.p, B.col.p, Bx, By, n_in, coef, X,
                                                               ldx, Y, ldy, coff, ncol);
    LAUNCH_CHECK(c);
}
void spmm_grad(tt_ctx* c, const Csr& BT, const double* BTx, const double* BTy, double coef, const double* X,
               int ldx, double* Y, int ldy, int coff, int ncol) {
    const long long threads = 2LL * BT.n_rows * 32;
    k_spmm_grad<<<ceil_div(threads, 256), 256, 0, c->stream>>>(BT.n_rows, BT.rowptr.p, BT.col.p, BTx, BTy, coef, X,
                                                                ldx, Y, ldy, coff, ncol);
    LAUNCH_CHECK(c);
}

// ============================================================== banded LU
namespace {
__global__ void __launch_bounds__(1024) k_band_factor(double* __restrict__ ab, int n, int bw, int* status) {
    const int W = 2 * bw + 1;
    extern __shared__ double lmul[];
    for (int k = 0; k < n; ++k) {
        const int nr = min(bw, n - 1 - k);
        const double piv = ab[(size_t)k * W + bw];
        if (piv == 0.0 || !(piv == piv)) {
            if (threadIdx.x == 0) atomicExch(status, DEV_NAN);
            return;
        }
        for (int r = threadIdx.x; r < nr; r += blockDim.x) {
            const int i = k + 1 + r;
            const double l = ab[(size_t)i * W + (k - i + bw)] / piv;
            ab[(size_t)i * W + (k - i + bw)] = l;
            lmul[r] = l;
        }
        __syncthreads();
        const int tot = nr * nr;
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int r = e / nr, cc = e % nr;
            const int i = k + 1 + r, j = k + 1 + cc;
            ab[(size_t)i * W + (j - i + bw)] -= lmul[r] * ab[(size_t)k * W + (j - k + bw)];
        }
        __syncthreads();
    }
}

template <typename TC>
__global__ void k_band_solve(const double* __restrict__ ab, int n, int bw, double* __restrict__ X, int ldx,
                             int ncol, int ncomp) {
    extern __shared__ __align__(16) unsigned char xs_raw[];
    TC* xs = reinterpret_cast<TC*>(xs_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int job = blockIdx.x * nw + warp;
    if (job >= ncol * ncomp) return;
    const int comp = job / ncol, b = job % ncol;
    TC* x = xs + (size_t)warp * n;
    const int W = 2 * bw + 1;
    for (int i = lane; i < n; i += 32) x[i] = TC(X[((size_t)comp * n + i) * ldx + b]);
    __syncwarp();
    for (int i = 0; i < n; ++i) {
        const int j0 = max(0, i - bw);
        TC s = TC(0);
        for (int j = j0 + lane; j < i; j += 32) s = fma(TC(ab[(size_t)i * W + j - i + bw]), x[j], s);
        s = warp_sum(s);
        if (lane == 0) x[i] -= s;
        __syncwarp();
    }
    for (int i = n - 1; i >= 0; --i) {
        const int j1 = min(n - 1, i + bw);
        TC s = TC(0);
        for (int j = i + 1 + lane; j <= j1; j += 32) s = fma(TC(ab[(size_t)i * W + j - i + bw]), x[j], s);
        s = warp_sum(s);
        if (lane == 0) x[i] = (x[i] - s) / TC(ab[(size_t)i * W + bw]);
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) X[((size_t)comp * n + i) * ldx + b] = (double)x[i];
}
}  // namespace

void band_factor(tt_ctx* c, double* ab, int n, int bw) {
    const size_t smem = (size_t)std::max(bw, 1) * sizeof(double);
    ProfScope prof(c, PROF_BAND_FACTOR, 2.0 * n * bw * bw, 16.0 * n * (2 * bw + 1));
    k_band_factor<<<1, 1024, smem, c->stream>>>(ab, n, bw, c->dstatus);
    LAUNCH_CHECK(c);
}

void band_solve(tt_ctx* c, const double* ab, int n, int bw, double* X, int ldx, int ncol, int ncomp) {
    const size_t per = (size_t)n * (c->fast ? sizeof(float) : sizeof(double));
    int nw = (int)std::max<size_t>(1, std::min<size_t>(8, (200 * 1024) / per));
    const int jobs = ncol * ncomp;
    // forward + backward substitution: 2 * 2 n bw flops per column; band read once, columns in and out
    ProfScope prof(c, PROF_BAND_SOLVE, 4.0 * n * bw * jobs, 8.0 * n * (2 * bw + 1) + 16.0 * n * jobs);
    nw = std::min(nw, std::max(1, jobs));
    auto kern = c->fast ? k_band_solve<float> : k_band_solve<double>;
    CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    kern<<<ceil_div(jobs, nw), 32 * nw, per * nw, c->stream>>>(ab, n, bw, X, ldx, ncol, ncomp);
    LAUNCH_CHECK(c);
}

// ============================================================== assembly drivers
static void build_gather(const std::vector<std::vector<std::pair<int, int>>>& contrib_by_row,
                         const std::vector<std::vector<int>>& cols, Csr& csr, Gather& g, int n_cols, tt_ctx* c) {
    // contrib_by_row[row] = list of (col, local index)
    const int n = (int)cols.size();
    std::vector<int> rp(n + 1, 0), cl;
    for (int i = 0; i < n; ++i) rp[i + 1] = rp[i] + (int)cols[i].size();
    cl.reserve(rp[n]);
    for (int i = 0; i < n; ++i) cl.insert(cl.end(), cols[i].begin(), cols[i].end());
    const int nnz = rp[n];
    std::vector<std::vector<int>> per(nnz);
    for (int i = 0; i < n; ++i)
        for (auto& pr : contrib_by_row[i]) {
            const auto it = std::lower_bound(cols[i].begin(), cols[i].end(), pr.first);
            per[rp[i] + (int)(it - cols[i].begin())].push_back(pr.second);
        }
    std::vector<int> gp(nnz + 1, 0), gi;
    for (int s = 0; s < nnz; ++s) {
        std::sort(per[s].begin(), per[s].end());
        gp[s + 1] = gp[s] + (int)per[s].size();
        gi.insert(gi.end(), per[s].begin(), per[s].end());
    }
    csr.n_rows = n; csr.n_cols = n_cols; csr.nnz = nnz;
    csr.rowptr.alloc(c, n + 1);
    csr.col.alloc(c, std::max(nnz, 1));
    g.ptr.alloc(c, nnz + 1);
    g.idx.alloc(c, std::max<size_t>(gi.size(), 1));
    CUDA_CHECK(cudaMemcpyAsync(csr.rowptr.p, rp.data(), rp.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    if (nnz) CUDA_CHECK(cudaMemcpyAsync(csr.col.p, cl.data(), cl.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CUDA_CHECK(cudaMemcpyAsync(g.ptr.p, gp.data(), gp.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    if (!gi.empty()) CUDA_CHECK(cudaMemcpyAsync(g.idx.p, gi.data(), gi.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CUDA_CHECK(cudaStreamSynchronize(c->stream));   // host vectors go out of scope
}

static void gather_vals(tt_ctx* c, const Csr& csr, const Gather& g, int nf, long long L, const double* loc,
                        double* vals) {
    if (csr.nnz == 0) return;
    const long long tot = (long long)csr.nnz * nf;
    k_gather<<<ceil_div(tot, 256), 256, 0, c->stream>>>(csr.nnz, nf, L, g.ptr.p, g.idx.p, loc, vals);
    LAUNCH_CHECK(c);
}

void assemble_conv(tt_ctx* c, tt_problem* P, const double* W, int ldw, int nf, double* vals_ff, double* vals_fD) {
    if (nf <= 0) return;
    DBuf<double> loc(c, (size_t)nf * P->n_elem * 81);
    k_local_conv<<<dim3(P->n_elem, nf), 96, 0, c->stream>>>(P->n_elem, P->n_nodes, P->h, P->eq2.p, W, ldw, loc.p);
    LAUNCH_CHECK(c);
    gather_vals(c, P->ff, P->g_ff, nf, (long long)P->n_elem * 81, loc.p, vals_ff);
    if (vals_fD) gather_vals(c, P->fD, P->g_fD, nf, (long long)P->n_elem * 81, loc.p, vals_fD);
}

void assemble_pconv(tt_ctx* c, tt_problem* P, const double* W, int ldw, int nf, double* vals_pp) {
    if (nf <= 0) return;
    DBuf<double> loc(c, (size_t)nf * P->n_elem * 16);
    k_local_pconv<<<dim3(P->n_elem, nf), 32, 0, c->stream>>>(P->n_elem, P->n_nodes, P->h, P->eq2.p, W, ldw, loc.p);
    LAUNCH_CHECK(c);
    gather_vals(c, P->pp, P->g_pp, nf, (long long)P->n_elem * 16, loc.p, vals_pp);
}

void scatter_band(tt_ctx* c, tt_problem* P, const double* vals, double* ab) {
    k_scatter_band<<<ceil_div(P->n_v, 256), 256, 0, c->stream>>>(P->n_v, P->bwK, P->ff.rowptr.p, P->ff.col.p, vals, ab);
    LAUNCH_CHECK(c);
}

void assemble_K_vals(tt_ctx* c, tt_problem* P, const double* wfield, double* kv) {
    const int nnz = P->ff.nnz;
    DBuf<double> nv;
    if (wfield) {
        nv.alloc(c, nnz);
        assemble_conv(c, P, wfield, 1, 1, nv.p, nullptr);
    }
    k_axpy3<<<ceil_div(nnz, 256), 256, 0, c->stream>>>(nnz, 1.0 / P->tau, P->M_ff.p, P->A_ff.p, nv.p, kv);
    LAUNCH_CHECK(c);
}

void assemble_K_band(tt_ctx* c, tt_problem* P, const double* wfield, double* ab) {
    DBuf<double> kv(c, P->ff.nnz);
    assemble_K_vals(c, P, wfield, kv.p);
    fill_zero(c, ab, (size_t)P->n_v * (2 * P->bwK + 1));
    scatter_band(c, P, kv.p, ab);
    band_factor(c, ab, P->n_v, P->bwK);
}

// ============================================================== gPC (Section 3.2)
// Gauss-Legendre nodes on [-1, 1] by Newton's method on P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0); w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) { const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            const double pn = n == 1 ? z : p1, pnm1 = n == 1 ? 1.0 : p0;
            const double dp = n * (z * pn - pnm1) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) { const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
        const double pn = n == 1 ? z : p1, pnm1 = n == 1 ? 1.0 : p0;
        const double dp = n * (z * pn - pnm1) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// orthonormal Legendre for U(-sqrt3, sqrt3) evaluated at t = xi / sqrt3
static double pn_scaled(int n, double t) {
    double p0 = 1.0, p1 = t;
    if (n == 0) return 1.0;
    for (int k = 2; k <= n; ++k) { const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
    return std::sqrt(2.0 * n + 1.0) * p1;
}

static void gpc_tables(int m, int n_xi, const long long* mi, std::vector<double>& G, std::vector<double>& H) {
    int dmax = 0;
    for (int i = 0; i < n_xi * m; ++i) dmax = std::max(dmax, (int)mi[i]);
    const int D = dmax + 2;
    std::vector<double> x, w;
    gauss_legendre(3 * D + 4, x, w);
    std::vector<double> T((size_t)D * D * D, 0.0), X((size_t)D * D, 0.0);
    for (size_t q = 0; q < x.size(); ++q) {
        const double wq = 0.5 * w[q];
        std::vector<double> pv(D);
        for (int a = 0; a < D; ++a) pv[a] = pn_scaled(a, x[q]);
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b) {
                X[a * D + b] += wq * std::sqrt(3.0) * x[q] * pv[a] * pv[b];
                for (int cc = 0; cc < D; ++cc) T[((size_t)a * D + b) * D + cc] += wq * pv[a] * pv[b] * pv[cc];
            }
    }
    G.assign((size_t)(m + 1) * n_xi * n_xi, 0.0);
    for (int r = 0; r < n_xi; ++r) G[(size_t)r * n_xi + r] = 1.0;
    for (int l = 0; l < m; ++l)
        for (int r = 0; r < n_xi; ++r)
            for (int s = 0; s < n_xi; ++s) {
                bool same = true;
                for (int k = 0; k < m; ++k)
                    if (k != l && mi[r * m + k] != mi[s * m + k]) same = false;
                G[((size_t)(l + 1) * n_xi + r) * n_xi + s] = same ? X[mi[r * m + l] * D + mi[s * m + l]] : 0.0;
            }
    H.assign((size_t)n_xi * n_xi * n_xi, 1.0);
    for (int l = 0; l < n_xi; ++l)
        for (int r = 0; r < n_xi; ++r)
            for (int s = 0; s < n_xi; ++s) {
                double v = 1.0;
                for (int k = 0; k < m; ++k)
                    v *= T[((size_t)mi[l * m + k] * D + mi[r * m + k]) * D + mi[s * m + k]];
                H[((size_t)l * n_xi + r) * n_xi + s] = v;
            }
}

// ============================================================== problem build
void build_problem(tt_ctx* c, tt_problem* P, const tt_problem_desc* d) {
    TT_REQUIRE(d && d->n_nodes > 0 && d->n_elem > 0 && d->n_pnodes > 0 && d->n_t > 0 && d->n_xi > 0 && d->m >= 0,
               "bad problem description");
    TT_REQUIRE(d->xy && d->elem_q2 && d->elem_q1 && d->dirichlet && d->inflow && d->nu && d->tprofile,
               "problem description has null arrays");
    TT_REQUIRE(d->m == 0 || d->multi_index, "multi_index missing");
    upload_tables();
    P->ctx = c;
    P->n_nodes = d->n_nodes; P->n_elem = d->n_elem; P->n_p = d->n_pnodes;
    P->m = d->m; P->n_xi = d->n_xi; P->n_t = d->n_t; P->tau = d->tau; P->h = d->h;
    const int n = d->n_nodes, E = d->n_elem, np_ = d->n_pnodes;
    P->hxy.assign(d->xy, d->xy + 2 * (size_t)n);
    P->fidx.assign(n, -1);
    P->didx.assign(n, -1);
    int nf = 0, nd = 0;
    for (int i = 0; i < n; ++i) {
        if (d->dirichlet[i]) P->didx[i] = nd++; else P->fidx[i] = nf++;
    }
    P->n_v = nf; P->n_D = nd;
    TT_REQUIRE(nf > 0, "no free velocity nodes");
    std::vector<int> q2((size_t)E * 9), q1((size_t)E * 4);
    for (size_t i = 0; i < q2.size(); ++i) {
        TT_REQUIRE(d->elem_q2[i] >= 0 && d->elem_q2[i] < n, "elem_q2 index out of range");
        q2[i] = (int)d->elem_q2[i];
    }
    for (size_t i = 0; i < q1.size(); ++i) {
        TT_REQUIRE(d->elem_q1[i] >= 0 && d->elem_q1[i] < np_, "elem_q1 index out of range");
        q1[i] = (int)d->elem_q1[i];
    }
    for (int i = 0; i < d->n_xi; ++i) {
        int deg = 0;
        for (int k = 0; k < d->m; ++k) deg += (int)d->multi_index[i * d->m + k];
        TT_REQUIRE(i != 0 || deg == 0, "multi-index 0 must be the constant polynomial");
    }
    P->eq2.alloc(c, q2.size());
    P->eq1.alloc(c, q1.size());
    CUDA_CHECK(cudaMemcpyAsync(P->eq2.p, q2.data(), q2.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CUDA_CHECK(cudaMemcpyAsync(P->eq1.p, q1.data(), q1.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    P->node_free.alloc(c, n);
    P->node_dir.alloc(c, n);
    CUDA_CHECK(cudaMemcpyAsync(P->node_free.p, P->fidx.data(), n * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CUDA_CHECK(cudaMemcpyAsync(P->node_dir.p, P->didx.data(), n * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    {
        std::vector<int> fl, dl;
        for (int i = 0; i < n; ++i) (P->fidx[i] >= 0 ? fl : dl).push_back(i);
        P->free_nodes.alloc(c, std::max<size_t>(1, fl.size()));
        P->dir_nodes.alloc(c, std::max<size_t>(1, dl.size()));
        CUDA_CHECK(cudaMemcpyAsync(P->free_nodes.p, fl.data(), fl.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        if (!dl.empty())
            CUDA_CHECK(cudaMemcpyAsync(P->dir_nodes.p, dl.data(), dl.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
    }

    // ---- patterns and gather maps
    std::vector<std::vector<int>> cff(nf), cfD(nf), cBF(np_), cBD(np_), cpp(np_);
    std::vector<std::vector<std::pair<int, int>>> lff(nf), lfD(nf), lBF(np_), lBD(np_), lpp(np_);
    for (int e = 0; e < E; ++e) {
        for (int i = 0; i < 9; ++i) {
            const int ri = P->fidx[q2[e * 9 + i]];
            if (ri < 0) continue;
            for (int j = 0; j < 9; ++j) {
                const int nj = q2[e * 9 + j];
                if (P->fidx[nj] >= 0) { cff[ri].push_back(P->fidx[nj]); lff[ri].push_back({P->fidx[nj], e * 81 + i * 9 + j}); }
                else { cfD[ri].push_back(P->didx[nj]); lfD[ri].push_back({P->didx[nj], e * 81 + i * 9 + j}); }
            }
        }
        for (int p = 0; p < 4; ++p)
            for (int p2 = 0; p2 < 4; ++p2) {
                cpp[q1[e * 4 + p]].push_back(q1[e * 4 + p2]);
                lpp[q1[e * 4 + p]].push_back({q1[e * 4 + p2], e * 16 + p * 4 + p2});
            }
        for (int p = 0; p < 4; ++p) {
            const int rp = q1[e * 4 + p];
            for (int j = 0; j < 9; ++j) {
                const int nj = q2[e * 9 + j];
                if (P->fidx[nj] >= 0) { cBF[rp].push_back(P->fidx[nj]); lBF[rp].push_back({P->fidx[nj], e * 36 + p * 9 + j}); }
                else { cBD[rp].push_back(P->didx[nj]); lBD[rp].push_back({P->didx[nj], e * 36 + p * 9 + j}); }
            }
        }
    }
    auto uniq = [](std::vector<std::vector<int>>& v) {
        for (auto& r : v) { std::sort(r.begin(), r.end()); r.erase(std::unique(r.begin(), r.end()), r.end()); }
    };
    uniq(cff); uniq(cfD); uniq(cBF); uniq(cBD); uniq(cpp);
    build_gather(lff, cff, P->ff, P->g_ff, nf, c);
    build_gather(lfD, cfD, P->fD, P->g_fD, nd, c);
    build_gather(lBF, cBF, P->BF, P->g_BF, nf, c);
    build_gather(lBD, cBD, P->BD, P->g_BD, nd, c);
    build_gather(lpp, cpp, P->pp, P->g_pp, np_, c);
    {
        // diagonal slots of the pressure pattern
        std::vector<int> dslot(np_), prp(np_ + 1, 0);
        for (int i = 0; i < np_; ++i) prp[i + 1] = prp[i] + (int)cpp[i].size();
        for (int i = 0; i < np_; ++i) {
            const auto it = std::lower_bound(cpp[i].begin(), cpp[i].end(), i);
            TT_REQUIRE(it != cpp[i].end() && *it == i, "missing diagonal in the pressure pattern");
            dslot[i] = prp[i] + (int)(it - cpp[i].begin());
        }
        P->pdiag_slot.alloc(c, np_);
        CUDA_CHECK(cudaMemcpyAsync(P->pdiag_slot.p, dslot.data(), np_ * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
    }
    // bandwidths
    int bw = 0;
    for (int i = 0; i < nf; ++i)
        for (int j : cff[i]) bw = std::max(bw, std::abs(i - j));
    P->bwK = bw;
    // B^T (free velocity rows x pressure cols) with the slot permutation
    {
        std::vector<int> brp(np_ + 1, 0);
        for (int p = 0; p < np_; ++p) brp[p + 1] = brp[p] + (int)cBF[p].size();
        std::vector<std::vector<std::pair<int, int>>> rows(nf);
        for (int p = 0; p < np_; ++p)
            for (size_t t = 0; t < cBF[p].size(); ++t) rows[cBF[p][t]].push_back({p, brp[p] + (int)t});
        std::vector<int> rp(nf + 1, 0), cl, perm;
        int bwl = 0;
        for (int j = 0; j < nf; ++j) {
            std::sort(rows[j].begin(), rows[j].end());
            rp[j + 1] = rp[j] + (int)rows[j].size();
            for (auto& pr : rows[j]) { cl.push_back(pr.first); perm.push_back(pr.second); }
            for (auto& a : rows[j])
                for (auto& b : rows[j]) bwl = std::max(bwl, std::abs(a.first - b.first));
        }
        P->bwL = bwl;
        P->BT.n_rows = nf; P->BT.n_cols = np_; P->BT.nnz = rp[nf];
        P->BT.rowptr.alloc(c, nf + 1);
        P->BT.col.alloc(c, std::max(1, rp[nf]));
        P->bt_perm.alloc(c, std::max(1, rp[nf]));
        CUDA_CHECK(cudaMemcpyAsync(P->BT.rowptr.p, rp.data(), rp.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        CUDA_CHECK(cudaMemcpyAsync(P->BT.col.p, cl.data(), cl.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        CUDA_CHECK(cudaMemcpyAsync(P->bt_perm.p, perm.data(), perm.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        // diagonal slots of ff
        std::vector<int> dslot(nf);
        std::vector<int> frp(nf + 1, 0);
        for (int i = 0; i < nf; ++i) frp[i + 1] = frp[i] + (int)cff[i].size();
        for (int i = 0; i < nf; ++i) {
            const auto it = std::lower_bound(cff[i].begin(), cff[i].end(), i);
            TT_REQUIRE(it != cff[i].end() && *it == i, "missing diagonal in the velocity pattern");
            dslot[i] = frp[i] + (int)(it - cff[i].begin());
        }
        P->diag_slot.alloc(c, nf);
        CUDA_CHECK(cudaMemcpyAsync(P->diag_slot.p, dslot.data(), nf * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
    }

    // ---- values
    const int m1 = d->m + 1;
    P->nu.alloc(c, (size_t)m1 * np_);
    CUDA_CHECK(cudaMemcpyAsync(P->nu.p, d->nu, (size_t)m1 * np_ * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    {
        DBuf<double> loc(c, (size_t)E * 81);
        k_local_mass<<<E, 96, 0, c->stream>>>(E, P->h, loc.p);
        LAUNCH_CHECK(c);
        P->M_ff.alloc(c, std::max(1, P->ff.nnz));
        P->M_fD.alloc(c, std::max(1, P->fD.nnz));
        gather_vals(c, P->ff, P->g_ff, 1, (long long)E * 81, loc.p, P->M_ff.p);
        gather_vals(c, P->fD, P->g_fD, 1, (long long)E * 81, loc.p, P->M_fD.p);
    }
    {
        DBuf<double> loc(c, (size_t)m1 * E * 81);
        k_local_stiff<<<dim3(E, m1), 96, 0, c->stream>>>(E, np_, P->eq1.p, P->nu.p, loc.p);
        LAUNCH_CHECK(c);
        P->A_ff.alloc(c, (size_t)m1 * std::max(1, P->ff.nnz));
        P->A_fD.alloc(c, (size_t)m1 * std::max(1, P->fD.nnz));
        gather_vals(c, P->ff, P->g_ff, m1, (long long)E * 81, loc.p, P->A_ff.p);
        gather_vals(c, P->fD, P->g_fD, m1, (long long)E * 81, loc.p, P->A_fD.p);
    }
    {
        DBuf<double> loc(c, (size_t)2 * E * 36);
        k_local_div<<<dim3(E, 2), 64, 0, c->stream>>>(E, P->h, loc.p);
        LAUNCH_CHECK(c);
        DBuf<double> bf(c, (size_t)2 * std::max(1, P->BF.nnz)), bd(c, (size_t)2 * std::max(1, P->BD.nnz));
        gather_vals(c, P->BF, P->g_BF, 2, (long long)E * 36, loc.p, bf.p);
        gather_vals(c, P->BD, P->g_BD, 2, (long long)E * 36, loc.p, bd.p);
        P->Bx_F.alloc(c, std::max(1, P->BF.nnz)); P->By_F.alloc(c, std::max(1, P->BF.nnz));
        P->Bx_D.alloc(c, std::max(1, P->BD.nnz)); P->By_D.alloc(c, std::max(1, P->BD.nnz));
        CUDA_CHECK(cudaMemcpyAsync(P->Bx_F.p, bf.p, P->BF.nnz * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        CUDA_CHECK(cudaMemcpyAsync(P->By_F.p, bf.p + P->BF.nnz, P->BF.nnz * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        if (P->BD.nnz) {
            CUDA_CHECK(cudaMemcpyAsync(P->Bx_D.p, bd.p, P->BD.nnz * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
            CUDA_CHECK(cudaMemcpyAsync(P->By_D.p, bd.p + P->BD.nnz, P->BD.nnz * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        }
        P->BTx.alloc(c, std::max(1, P->BT.nnz)); P->BTy.alloc(c, std::max(1, P->BT.nnz));
        k_take<<<ceil_div(P->BT.nnz, 256), 256, 0, c->stream>>>(P->BT.nnz, P->bt_perm.p, P->Bx_F.p, P->BTx.p);
        LAUNCH_CHECK(c);
        k_take<<<ceil_div(P->BT.nnz, 256), 256, 0, c->stream>>>(P->BT.nnz, P->bt_perm.p, P->By_F.p, P->BTy.p);
        LAUNCH_CHECK(c);
    }
    {
        // pressure-space mass and mean diffusion (Section 5.2), and M_p* = diag(M_p)
        DBuf<double> loc(c, (size_t)2 * E * 16);
        k_local_pmat<<<dim3(E, 2), 32, 0, c->stream>>>(E, np_, P->h, P->eq1.p, P->nu.p, loc.p);
        LAUNCH_CHECK(c);
        DBuf<double> pv(c, (size_t)2 * std::max(1, P->pp.nnz));
        gather_vals(c, P->pp, P->g_pp, 2, (long long)E * 16, loc.p, pv.p);
        P->Mp_pp.alloc(c, std::max(1, P->pp.nnz));
        P->Ap_pp.alloc(c, std::max(1, P->pp.nnz));
        CUDA_CHECK(cudaMemcpyAsync(P->Mp_pp.p, pv.p, P->pp.nnz * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        CUDA_CHECK(cudaMemcpyAsync(P->Ap_pp.p, pv.p + P->pp.nnz, P->pp.nnz * sizeof(double), cudaMemcpyDeviceToDevice,
                                   c->stream));
        P->Mpstar.alloc(c, np_);
        k_take<<<ceil_div(np_, 256), 256, 0, c->stream>>>(np_, P->pdiag_slot.p, P->Mp_pp.p, P->Mpstar.p);
        LAUNCH_CHECK(c);
    }
    P->Mstar.alloc(c, nf);
    k_take<<<ceil_div(nf, 256), 256, 0, c->stream>>>(nf, P->diag_slot.p, P->M_ff.p, P->Mstar.p);
    LAUNCH_CHECK(c);
    // pressure Laplacian B M*^-1 B^T, factorised once
    P->Lp_band.alloc(c, (size_t)np_ * (2 * P->bwL + 1));
    fill_zero(c, P->Lp_band.p, (size_t)np_ * (2 * P->bwL + 1));
    k_lp_band<<<ceil_div(np_, 128), 128, 0, c->stream>>>(np_, P->bwL, P->BF.rowptr.p, P->BF.col.p, P->Bx_F.p, P->By_F.p,
                                                          P->BT.rowptr.p, P->BT.col.p, P->BTx.p, P->BTy.p,
                                                          P->Mstar.p, P->Lp_band.p);
    LAUNCH_CHECK(c);
    band_factor(c, P->Lp_band.p, np_, P->bwL);

    // ---- gPC
    std::vector<double> G, H;
    gpc_tables(d->m, d->n_xi, d->multi_index, G, H);
    P->hG = G;
    P->G.alloc(c, G.size());
    P->H.alloc(c, H.size());
    CUDA_CHECK(cudaMemcpyAsync(P->G.p, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_CHECK(cudaMemcpyAsync(P->H.p, H.data(), H.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));

    // ---- lifting u_D: ramp (x) psi_1 (x) boundary values (x1 comps, then x2 comps = 0)
    if (nd > 0) {
        std::vector<double> z3(2 * nd, 0.0), z2(d->n_xi, 0.0);
        for (int i = 0; i < n; ++i)
            if (P->didx[i] >= 0) z3[P->didx[i]] = d->inflow[i];
        z2[0] = 1.0;
        P->uD = tt_alloc(c, d->n_t, d->n_xi, 2 * nd, 1, 1);
        CUDA_CHECK(cudaMemcpyAsync(P->uD->z1, d->tprofile, d->n_t * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CUDA_CHECK(cudaMemcpyAsync(P->uD->z2, z2.data(), z2.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CUDA_CHECK(cudaMemcpyAsync(P->uD->z3, z3.data(), z3.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    }
    CUDA_CHECK(cudaStreamSynchronize(c->stream));
    check_status(c);
}

}  // namespace tt

tt_problem::~tt_problem() {
    tt::tt_free(uD);
    tt::tt_free(fu);
    tt::tt_free(fp);
}
