// Dense FP64 kernels of the TT rounding (Section 4.1).
//
//  * gemm: 64x64x16 tiles with arbitrary strides; split-K over the grid when the
//    output has few tiles, because GB300's FP64 pipe is narrow per SM and a
//    small product must still spread over every SM.
//  * qr_r: R factor of a tall n x c matrix by Householder reflections, one
//    cooperative launch.  Each CTA keeps a block of rows resident (shared
//    memory when it fits) and, per column, the CTAs exchange partial norms and
//    partial reflector dots through global memory across bounded grid
//    barriers (a flat-tree TSQR in which the tree is one reduction level).
//  * left_svd: R factor of A^T, then one-sided (Hestenes) Jacobi on R^T,
//    columns rotated pairwise in round-robin order, one warp per pair, one grid
//    barrier per round.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include <cooperative_groups.h>

#include "la.cuh"

namespace tt {

// ============================================================== GEMM
namespace {
constexpr int GB_M = 64, GB_N = 64, GB_K = 16;

template <typename TC>
__global__ void __launch_bounds__(256)
k_gemm(int M, int N, int K, double alpha, const double* __restrict__ A, long long as0,
       long long as1, const double* __restrict__ B, long long bs0, long long bs1, double beta,
       double* __restrict__ C, long long cs0, long long cs1, int kchunk, double* __restrict__ part) {
    __shared__ TC As[GB_K][GB_M + 1];
    __shared__ TC Bs[GB_K][GB_N + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.y * GB_M, j0 = blockIdx.x * GB_N;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    TC acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = TC(0);
    const bool a_rowfast = (as1 == 1);   // k contiguous: iterate k fastest
    const bool b_colfast = (bs1 == 1);   // j contiguous: iterate j fastest
    for (int k0 = kbeg; k0 < kend; k0 += GB_K) {
        for (int e = tid; e < GB_M * GB_K; e += 256) {
            int ii, kk;
            if (a_rowfast) { kk = e % GB_K; ii = e / GB_K; } else { ii = e % GB_M; kk = e / GB_M; }
            const int gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < M && gk < kend) ? TC(A[gi * as0 + gk * as1]) : TC(0);
        }
        for (int e = tid; e < GB_K * GB_N; e += 256) {
            int jj, kk;
            if (b_colfast) { jj = e % GB_N; kk = e / GB_N; } else { kk = e % GB_K; jj = e / GB_K; }
            const int gj = j0 + jj, gk = k0 + kk;
            Bs[kk][jj] = (gj < N && gk < kend) ? TC(B[gk * bs0 + gj * bs1]) : TC(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GB_K; ++kk) {
            TC av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int gi = i0 + ty * 4 + a;
        if (gi >= M) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int gj = j0 + tx * 4 + b;
            if (gj >= N) continue;
            const double v = (double)acc[a][b];
            if (part) {
                part[((size_t)blockIdx.z * M + gi) * N + gj] = v;
            } else {
                double* cp = C + gi * cs0 + gj * cs1;
                *cp = beta == 0.0 ? alpha * v : alpha * v + beta * *cp;
            }
        }
    }
}

__global__ void k_gemm_reduce(int M, int N, int S, double alpha, const double* __restrict__ part,
                              double beta, double* __restrict__ C, long long cs0, long long cs1) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)M * N) return;
    const int i = (int)(idx / N), j = (int)(idx % N);
    double s = 0.0;
    for (int z = 0; z < S; ++z) s += part[(size_t)z * M * N + idx];
    double* cp = C + i * cs0 + j * cs1;
    *cp = beta == 0.0 ? alpha * s : alpha * s + beta * *cp;
}
}  // namespace

void gemm(tt_ctx* c, int M, int N, int K, double alpha, MatView A, MatView B, double beta,
          MatViewMut C) {
    gemm_ws(c, M, N, K, alpha, A, B, beta, C, nullptr, 0);
}

void gemm_ws(tt_ctx* c, int M, int N, int K, double alpha, MatView A, MatView B, double beta,
             MatViewMut C, double* ws, size_t ws_len) {
    if (M <= 0 || N <= 0) return;
    if (K <= 0) {
        // C = beta C
        if (beta == 0.0) {
            copy_mat(c, M, N, MatView{C.p, C.s0, C.s1}, C, 0.0);
        } else if (beta != 1.0) {
            copy_mat(c, M, N, MatView{C.p, C.s0, C.s1}, C, beta);
        }
        return;
    }
    const int tm = ceil_div(M, GB_M), tn = ceil_div(N, GB_N);
    const int tiles = tm * tn;
    int S = 1;
    const int target = 2 * c->nsm;
    if (tiles < target && K > 2 * GB_K) {
        S = std::min(ceil_div(target, tiles), ceil_div(K, 4 * GB_K));
        S = std::max(S, 1);
    }
    // with a caller workspace, split-K is limited to what fits in it
    if (ws && S > 1) S = std::max<long long>(1, std::min<long long>(S, (long long)(ws_len / ((size_t)M * N))));
    const int kchunk = ceil_div(ceil_div(K, S), GB_K) * GB_K;
    S = ceil_div(K, kchunk);
    dim3 grid(tn, tm, S);
    ProfScope prof(c, PROF_GEMM, 2.0 * M * N * K, 8.0 * ((double)M * K + (double)K * N + (double)M * N));
    auto kern = c->fast ? k_gemm<float> : k_gemm<double>;
    if (S == 1) {
        kern<<<grid, 256, 0, c->stream>>>(M, N, K, alpha, A.p, A.s0, A.s1, B.p, B.s0, B.s1, beta,
                                          C.p, C.s0, C.s1, kchunk, nullptr);
        LAUNCH_CHECK(c);
    } else {
        DBuf<double> own;
        double* part = ws;
        if (!part) {
            own.alloc(c, (size_t)S * M * N);
            part = own.p;
        }
        kern<<<grid, 256, 0, c->stream>>>(M, N, K, alpha, A.p, A.s0, A.s1, B.p, B.s0, B.s1, beta,
                                          C.p, C.s0, C.s1, kchunk, part);
        LAUNCH_CHECK(c);
        const long long tot = (long long)M * N;
        k_gemm_reduce<<<ceil_div(tot, 256), 256, 0, c->stream>>>(M, N, S, alpha, part, beta, C.p,
                                                                  C.s0, C.s1);
        LAUNCH_CHECK(c);
    }
}

// ============================================================== copies
namespace {
__global__ void k_copy_mat(int m, int n, const double* __restrict__ A, long long a0, long long a1,
                           double* __restrict__ B, long long b0, long long b1, double alpha) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)m * n) return;
    int i, j;
    if (b0 == 1) { i = (int)(idx % m); j = (int)(idx / m); } else { j = (int)(idx % n); i = (int)(idx / n); }
    B[i * b0 + j * b1] = alpha == 0.0 ? 0.0 : alpha * A[i * a0 + j * a1];
}
}  // namespace

void copy_mat(tt_ctx* c, int m, int n, MatView A, MatViewMut B, double alpha) {
    if (m <= 0 || n <= 0) return;
    const long long tot = (long long)m * n;
    k_copy_mat<<<ceil_div(tot, 256), 256, 0, c->stream>>>(m, n, A.p, A.s0, A.s1, B.p, B.s0, B.s1, alpha);
    LAUNCH_CHECK(c);
}

void fill_zero(tt_ctx* c, double* p, size_t n) {
    if (n) CUDA_CHECK(cudaMemsetAsync(p, 0, n * sizeof(double), c->stream));
}

// ============================================================== QR (R only)
namespace {
template <typename TC>
struct QRParams {
    int n, c, k, nb, nbp, L;
    const double* A;
    long long rs, cs;
    double* R;
    int ldr;
    TC* gwork;
    TC* part;    // [G][L] per-CTA partials of the combined reduction
    TC* sums;    // [L]
    unsigned* bar;
    int* status;
    const double* fnorm;   // ||A||_F^2 (FP32 arithmetic works on A / ||A||_F), or null
    const double* fro2;    // ||A||_F^2 (zero-column threshold)
    long long wait_limit;  // grid-barrier polls before DEV_TIMEOUT
};

template <typename TC>
__device__ TC block_sum(TC v, TC* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    TC s = TC(0);
    if (warp == 0) {
        s = lane < nw ? red[lane] : TC(0);
        s = warp_sum(s);
        if (lane == 0) red[0] = s;
    }
    __syncthreads();
    s = red[0];
    __syncthreads();
    return s;
}

// Per-CTA partials for column j over the resident rows i >= j:
//   out[0]       = sum a_ij^2
//   out[1 + l]   = sum a_ij a_il           (l > j)
//   out[1 + c + l] = a_jl (owner of row j) (l >= j), 0 elsewhere
template <typename TC>
__device__ void qr_partials(const QRParams<TC>& P, const TC* W, int j, int row0, int rows, TC* red, TC* out) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int ib = max(0, j - row0);
    const TC* wj = W + (size_t)j * P.nbp;
    TC ss = TC(0);
    for (int i = ib + tid; i < rows; i += blockDim.x) ss += wj[i] * wj[i];
    ss = block_sum(ss, red);
    if (tid == 0) out[0] = ss;
    for (int l = j + 1 + warp; l < P.c; l += nw) {
        const TC* wl = W + (size_t)l * P.nbp;
        TC d = TC(0);
        for (int i = ib + lane; i < rows; i += 32) d += wj[i] * wl[i];
        d = warp_sum(d);
        if (lane == 0) out[1 + l] = d;
    }
    const int jloc = j - row0;
    const bool own = jloc >= 0 && jloc < rows;
    for (int l = j + tid; l < P.c; l += blockDim.x) out[1 + P.c + l] = own ? W[(size_t)l * P.nbp + jloc] : TC(0);
}

// TC: arithmetic type (double, or float for the mixed path); input and R are FP64.
// Householder with one combined reduction per column: v^T a_l = a_j^T a_l - alpha a_jl
// lets the norm of column j, its products with the trailing columns and row j travel
// together, so each column costs two grid barriers (partials ready, sums ready).
template <typename TC, bool kCluster>
__global__ void __launch_bounds__(256) k_qr_r(QRParams<TC> P) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    TC* sm = reinterpret_cast<TC*>(sm_raw);
    const int g = blockIdx.x, G = gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int row0 = g * P.nb;
    const int rows = max(0, min(P.nb, P.n - row0));
    TC* red = sm;                                   // [32]
    TC* W = P.gwork ? P.gwork + (size_t)g * P.nbp * P.c : sm + 32;   // [c][nbp]
    TC* mypart = P.part + (size_t)g * P.L;
    // FP32 arithmetic runs on A / ||A||_F so no square overflows; R is scaled back
    double sc = 1.0;
    if (P.fnorm) {
        const double f = sqrt(__ldcg(P.fnorm));   // P.fnorm holds ||A||_F^2
        sc = (f > 0.0 && f < 1e300) ? f : 1.0;
    }
    const double inv = 1.0 / sc;
    // numerically zero column: remaining squared norm at most 1e-30 ||A||_F^2 (in the
    // scaled units of the working copy)
    const TC thr = TC(1e-30 * __ldcg(P.fro2) * inv * inv);
    for (int l = warp; l < P.c; l += nw)
        for (int i = lane; i < rows; i += 32)
            W[(size_t)l * P.nbp + i] = TC(P.A[(long long)(row0 + i) * P.rs + (long long)l * P.cs] * inv);
    __syncthreads();
    if (P.k > 0) qr_partials(P, W, 0, row0, rows, red, mypart);
    const int gw = g * nw + warp, TW = G * nw;
    for (int j = 0; j < P.k; ++j) {
        if (*(volatile int*)P.status == DEV_TIMEOUT) return;
        group_barrier<kCluster>(P.bar, G, P.status, P.wait_limit);
        // reduce-scatter of the live entries: 0, 1 + (j, c), 1 + c + [j, c)
        const int nd = P.c - j - 1, ne = P.c - j;
        for (int t = gw; t < 1 + nd + ne; t += TW) {
            const int idx = t == 0 ? 0 : (t <= nd ? 1 + j + t : 1 + P.c + j + (t - 1 - nd));
            TC s = TC(0);
            for (int q = lane; q < G; q += 32) s += __ldcg(P.part + (size_t)q * P.L + idx);
            s = warp_sum(s);
            if (lane == 0) P.sums[idx] = s;
        }
        group_barrier<kCluster>(P.bar, G, P.status, P.wait_limit);
        const TC ss = __ldcg(P.sums), x0 = __ldcg(P.sums + 1 + P.c + j);
        const int jloc = j - row0;
        const bool own = jloc >= 0 && jloc < rows;
        // numerically zero column (Householder steps on it would only shrink rounding
        // noise towards the underflow range, where 2 / v^T v overflows): R(j, :) is row j
        // as it stands
        if (ss <= thr) {
            if (own)
                for (int l = tid; l < P.c; l += blockDim.x)
                    P.R[(size_t)j * P.ldr + l] = l < j ? 0.0 : (double)W[(size_t)l * P.nbp + jloc] * sc;
        } else {
            const TC sigma = sqrt(ss);
            const TC alpha = x0 >= TC(0) ? -sigma : sigma;
            const TC v0 = x0 - alpha;
            const TC beta = TC(1) / (ss + fabs(x0) * sigma);    // 2 / v^T v
            const int ib = max(0, j - row0);
            const TC* wj = W + (size_t)j * P.nbp;
            for (int l = j + 1 + warp; l < P.c; l += nw) {
                const TC el = __ldcg(P.sums + 1 + P.c + l);
                const TC wl = beta * (__ldcg(P.sums + 1 + l) - alpha * el);
                TC* col = W + (size_t)l * P.nbp;
                for (int i = ib + lane; i < rows; i += 32) {
                    const TC vi = (row0 + i == j) ? v0 : wj[i];
                    col[i] -= vi * wl;
                }
                if (own && lane == 0) P.R[(size_t)j * P.ldr + l] = (double)(el - v0 * wl) * sc;
            }
            if (own)
                for (int l = tid; l <= j; l += blockDim.x)
                    P.R[(size_t)j * P.ldr + l] = l < j ? 0.0 : (double)alpha * sc;
        }
        __syncthreads();
        if (j + 1 < P.k) qr_partials(P, W, j + 1, row0, rows, red, mypart);
    }
}

// Householder R factor on one thread-block cluster of G <= 16 CTAs, CTA g holding rows
// [g nb, g nb + nb) of A in shared memory.  The same combined reduction per column as
// k_qr_r (|a_j|^2 over the live rows, a_j^T a_l and row j), but the partials stay in
// each CTA's shared memory (double-buffered by column parity) and every CTA sums the
// G partials of each entry it needs through distributed shared memory, so a column
// costs one hardware cluster barrier.  Inside a CTA the dot products run a group of
// lanes per trailing column over the CTA's rows and the rank-1 update one thread per
// entry, so no column waits on a chain of warp reductions.  Row j of the working rows
// becomes R(j, :) in place (the diagonal is stored after the update) and R is written
// at the end.  With perm set, column pivoting (Businger and Golub): step j first swaps
// in the trailing column of largest remaining norm (norms downdated by R(j, l)^2, the
// same values in every CTA), A P = Q R, and perm[j] is the original index of column j.
template <typename TC>
struct QRClParams {
    int n, c, k, nb, nbp, L;
    const double* A;
    long long rs, cs;
    double* R;
    int ldr;
    const double* fnorm;   // ||A||_F^2 (FP32 arithmetic works on A / ||A||_F), or null
    int* perm;             // column permutation (pivoting), or null
};

template <typename TC>
__global__ void __launch_bounds__(256) k_qr_cl(QRClParams<TC> P) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char sm_raw[];
    TC* sm = reinterpret_cast<TC*>(sm_raw);
    const int G = (int)cl.num_blocks(), g = (int)cl.block_rank();
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const int row0 = g * P.nb;
    const int rows = max(0, min(P.nb, P.n - row0));
    const int c = P.c, L = P.L;
    const bool pivot = P.perm != nullptr;
    TC* red = sm;                                  // [32]
    TC* part = red + 32;                           // [2][L] this CTA's partials
    TC* sums = part + 2 * L;                       // [L] reduced entries
    TC* wl = sums + L;                             // [c] update coefficients
    TC* nrm2 = wl + c;                             // [c] remaining squared column norms
    TC* W = nrm2 + c;                              // [c][nbp] this CTA's rows
    int* pidx = reinterpret_cast<int*>(W + (size_t)c * P.nbp);   // [c] column of origin
    int* ired = pidx + c;                          // [32] argmax indices
    double sc = 1.0;
    if (P.fnorm) {
        const double f = sqrt(__ldcg(P.fnorm));
        sc = (f > 0.0 && f < 1e300) ? f : 1.0;
    }
    const double inv = 1.0 / sc;
    // load: the unit-stride index of A runs over consecutive threads
    const long long tot = (long long)rows * c;
    if (P.cs == 1) {
        for (long long t = tid; t < tot; t += nt) {
            const int i = (int)(t / c), l = (int)(t % c);
            W[(size_t)l * P.nbp + i] = TC(P.A[(long long)(row0 + i) * P.rs + l] * inv);
        }
    } else {
        for (long long t = tid; t < tot; t += nt) {
            const int l = (int)(t / rows), i = (int)(t % rows);
            W[(size_t)l * P.nbp + i] = TC(P.A[(long long)(row0 + i) * P.rs + (long long)l * P.cs] * inv);
        }
    }
    __syncthreads();
    // column norms over all rows (pivot order) and ||A||_F^2 (zero-column threshold):
    // partials in buffer 1 (column 0 writes buffer 0, and no CTA writes buffer 1 before
    // every CTA has passed column 0's barrier)
    TC thr;
    {
        TC* np = part + L;
        for (int l = tid; l < c; l += nt) {
            const TC* w2 = W + (size_t)l * P.nbp;
            TC s = TC(0);
            for (int i = 0; i < rows; ++i) s += w2[i] * w2[i];
            np[l] = s;
            pidx[l] = l;
        }
        cl.sync();
        TC f = TC(0);
        for (int l = tid; l < c; l += nt) {
            TC s = TC(0);
            for (int q = 0; q < G; ++q) s += *cl.map_shared_rank(np + l, q);
            nrm2[l] = s;
            f += s;
        }
        f = warp_sum(f);
        if (lane == 0) red[warp] = f;
        __syncthreads();
        f = TC(0);
        for (int q = 0; q < (nt >> 5); ++q) f += red[q];
        // a column whose remaining squared norm is at most 1e-30 ||A||_F^2 is numerically
        // zero: Householder steps on such columns only shrink rounding noise further,
        // towards the underflow range where 2 / v^T v overflows
        thr = TC(1e-30) * f;
        __syncthreads();
    }
    for (int j = 0; j < P.k; ++j) {
        TC* mypart = part + (j & 1) * L;
        const int ib = max(0, j - row0);
        const int live = max(0, rows - ib);
        const int jloc = j - row0;
        const bool own = jloc >= 0 && jloc < rows;
        if (pivot) {
            // the trailing column of largest remaining norm (lowest index on ties)
            TC bv = TC(-1);
            int bi = c;
            for (int l = j + tid; l < c; l += nt) {
                const TC v = nrm2[l];
                if (v > bv) { bv = v; bi = l; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const TC ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            if (lane == 0) { red[warp] = bv; ired[warp] = bi; }
            __syncthreads();
            if (tid == 0) {
                for (int q = 1; q < (nt >> 5); ++q)
                    if (red[q] > bv || (red[q] == bv && ired[q] < bi)) { bv = red[q]; bi = ired[q]; }
                ired[0] = bi;
            }
            __syncthreads();
            const int pv = ired[0];
            if (pv != j && pv < c) {
                TC* a0 = W + (size_t)j * P.nbp;
                TC* a1 = W + (size_t)pv * P.nbp;
                for (int i = tid; i < rows; i += nt) {
                    const TC x = a0[i];
                    a0[i] = a1[i];
                    a1[i] = x;
                }
                if (tid == 0) {
                    const TC x = nrm2[j]; nrm2[j] = nrm2[pv]; nrm2[pv] = x;
                    const int y = pidx[j]; pidx[j] = pidx[pv]; pidx[pv] = y;
                }
            }
            __syncthreads();
        }
        const TC* wj = W + (size_t)j * P.nbp;
        // (a) partials: [0] = |a_j|^2, [1 + l] = a_j^T a_l (l > j), [1 + c + l] = a_jl (owner)
        {
            TC s = TC(0);
            for (int i = ib + tid; i < rows; i += nt) s += wj[i] * wj[i];
            s = warp_sum(s);
            if (lane == 0) red[warp] = s;
        }
        const int nl = c - j - 1;
        if (nl > 0) {
            int tpc = 1;                            // lanes per trailing column
            while (tpc < 32 && 2 * tpc * nl <= nt) tpc *= 2;
            const int per = nt / tpc;               // columns per pass
            for (int l0 = 0; l0 < nl; l0 += per) {
                const int l = j + 1 + l0 + tid / tpc, sub = tid % tpc;
                TC d0 = TC(0), d1 = TC(0);
                if (l < c) {
                    const TC* w2 = W + (size_t)l * P.nbp;
                    int i = ib + sub;
                    for (; i + tpc < rows; i += 2 * tpc) {
                        d0 += wj[i] * w2[i];
                        d1 += wj[i + tpc] * w2[i + tpc];
                    }
                    if (i < rows) d0 += wj[i] * w2[i];
                }
                TC d = d0 + d1;
                for (int o = tpc >> 1; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                if (sub == 0 && l < c) mypart[1 + l] = d;
            }
        }
        if (own)
            for (int l = j + tid; l < c; l += nt) mypart[1 + c + l] = W[(size_t)l * P.nbp + jloc];
        __syncthreads();
        if (tid < 32) {
            TC s = tid < (nt >> 5) ? red[tid] : TC(0);
            s = warp_sum(s);
            if (tid == 0) mypart[0] = s;
        }
        // (b) every CTA's partials are complete
        cl.sync();
        // (c) sums: the norm and the products over all CTAs, row j from its owner
        const int owner = min(j / P.nb, G - 1);
        for (int t = tid; t < 1 + nl + (c - j); t += nt) {
            if (t <= nl) {
                const int idx = t == 0 ? 0 : 1 + j + t;
                // all G remote loads in flight at once, then a fixed-order sum
                TC v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = q < G ? *cl.map_shared_rank(part + (j & 1) * L + idx, q) : TC(0);
#pragma unroll
                for (int w2 = 8; w2 > 0; w2 >>= 1)
#pragma unroll
                    for (int q = 0; q < w2; ++q) v[q] += v[q + w2];
                sums[idx] = v[0];
            } else {
                const int idx = 1 + c + j + (t - 1 - nl);
                sums[idx] = *cl.map_shared_rank(part + (j & 1) * L + idx, owner);
            }
        }
        __syncthreads();
        const TC ss = sums[0], x0 = sums[1 + c + j];
        // numerically zero column: row j stays as it stands
        if (ss <= thr) continue;
        const TC sigma = sqrt(ss);
        const TC alpha = x0 >= TC(0) ? -sigma : sigma;
        const TC v0 = x0 - alpha;
        const TC beta = TC(1) / (ss + fabs(x0) * sigma);    // 2 / v^T v
        // v = a_j - alpha e_j: v^T a_l = a_j^T a_l - alpha a_jl, w_l = beta v^T a_l;
        // R(j, l) = a_jl - v0 w_l leaves |R(j, l)|^2 of column l's remaining norm behind
        for (int l = j + 1 + tid; l < c; l += nt) {
            const TC el = sums[1 + c + l];
            const TC w = beta * (sums[1 + l] - alpha * el);
            wl[l] = w;
            if (pivot) {
                const TC r = el - v0 * w;
                nrm2[l] = max(TC(0), nrm2[l] - r * r);
            }
        }
        __syncthreads();
        // (d) a_l -= v w_l on this CTA's live rows, one thread per entry
        const long long upd = (long long)nl * live;
        for (long long t = tid; t < upd; t += nt) {
            const int l = j + 1 + (int)(t / live), i = ib + (int)(t % live);
            const TC vi = (row0 + i == j) ? v0 : wj[i];
            W[(size_t)l * P.nbp + i] -= vi * wl[l];
        }
        __syncthreads();
        if (own && tid == 0) W[(size_t)j * P.nbp + jloc] = alpha;
    }
    __syncthreads();
    // R(i, :) for the rows this CTA holds
    for (long long t = tid; t < (long long)rows * c; t += nt) {
        const int i = (int)(t / c), l = (int)(t % c);
        const int gi = row0 + i;
        if (gi < P.k) P.R[(size_t)gi * P.ldr + l] = l < gi ? 0.0 : (double)W[(size_t)l * P.nbp + i] * sc;
    }
    if (pivot && g == 0)
        for (int l = tid; l < c; l += nt) P.perm[l] = pidx[l];
    // no CTA leaves while another may still read its partials
    cl.sync();
}

// sum of squares of a strided n x cols matrix, accumulated into *out (zeroed by the caller)
__global__ void k_frob2_strided(int n, int cols, const double* __restrict__ A, long long rs, long long cs,
                                double* __restrict__ out) {
    double s = 0.0;
    const long long len = (long long)n * cols;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len; t += (long long)gridDim.x * blockDim.x) {
        const long long i = t % n, l = t / n;
        const double x = A[i * rs + l * cs];
        s = fma(x, x, s);
    }
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

// Returns whether the columns were pivoted (perm written): only the cluster kernel
// pivots; the grid kernel (rows beyond one cluster's shared memory) does not.
template <typename TC>
bool qr_r_launch(tt_ctx* c, int n, int cols, MatView A, double* R, int ldr, int* perm) {
    const int k = std::min(n, cols);
    const int L = 2 * cols + 1;
    DBuf<double> fn;
    if (sizeof(TC) < sizeof(double)) {
        fn.alloc(c, 1);
        CUDA_CHECK(cudaMemsetAsync(fn.p, 0, sizeof(double), c->stream));
        const long long len = (long long)n * cols;
        const int fb = (int)std::min<long long>(2LL * c->nsm, std::max(1LL, (len + 255) / 256));
        k_frob2_strided<<<fb, 256, 0, c->stream>>>(n, cols, A.p, A.s0, A.s1, fn.p);
        LAUNCH_CHECK(c);
    }
    // Householder R factor: 2 n c^2 - 2 c^3 / 3 flops (n >= c); reads A once, writes R
    const double kk = k;
    ProfScope prof(c, PROF_QR, 2.0 * kk * kk * ((double)n + cols - kk) - 2.0 * kk * kk * kk / 3.0,
                   8.0 * ((double)n * cols + kk * cols));
    {
        // one cluster of up to 16 CTAs with the rows in shared memory (at least 4 rows a
        // CTA: the FP64 work of a column spreads over as many SMs as the cluster has, at
        // one cluster barrier per column)
        const int Gc = std::min(16, std::max(1, ceil_div(n, 4)));
        const int nbc = ceil_div(n, Gc);
        const int Gu = ceil_div(n, nbc);
        const int nbpc = nbc | 1;
        const size_t smc = ((size_t)32 + 3 * (size_t)L + 2 * (size_t)cols + (size_t)cols * nbpc) * sizeof(TC) +
                           ((size_t)cols + 32) * sizeof(int);
        if (smc <= 200 * 1024) {
            CUDA_CHECK(cudaFuncSetAttribute(k_qr_cl<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
            if (Gu == 1 || max_cluster_ctas(c, (const void*)k_qr_cl<TC>, 256, smc) >= Gu) {
                QRClParams<TC> Q;
                Q.n = n; Q.c = cols; Q.k = k; Q.nb = nbc; Q.nbp = nbpc; Q.L = L;
                Q.A = A.p; Q.rs = A.s0; Q.cs = A.s1;
                Q.R = R; Q.ldr = ldr;
                Q.fnorm = fn.p;
                Q.perm = perm;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(Gu);
                cfg.blockDim = dim3(256);
                cfg.dynamicSmemBytes = smc;
                cfg.stream = c->stream;
                cudaLaunchAttribute attr;
                attr.id = cudaLaunchAttributeClusterDimension;
                attr.val.clusterDim.x = Gu;
                attr.val.clusterDim.y = 1;
                attr.val.clusterDim.z = 1;
                cfg.attrs = &attr;
                cfg.numAttrs = 1;
                CUDA_CHECK(cudaLaunchKernelEx(&cfg, k_qr_cl<TC>, Q));
                count_launch(c);
                return perm != nullptr;
            }
        }
    }
    int G = std::min(c->nsm, std::max(1, ceil_div(n, 16)));
    // Small panels run in one CTA: its columns then cost two block barriers instead
    // of two grid barriers (~2 us each), which dominate below ~4k (FP64: one SM's
    // FP64 rate is low) or ~48k (FP32) entries.
    const long long small_entries = sizeof(TC) < sizeof(double) ? 48 * 1024 : 4 * 1024;
    if ((long long)n * cols <= small_entries) G = 1;
    const int nb = ceil_div(n, G);
    G = ceil_div(n, nb);
    const int nbp = nb | 1;
    size_t smem = 32 * sizeof(TC);
    const size_t wbytes = (size_t)nbp * cols * sizeof(TC);
    DBuf<TC> gwork;
    const size_t smem_limit = 200 * 1024;
    if (smem + wbytes <= smem_limit) {
        smem += wbytes;
    } else {
        gwork.alloc(c, (size_t)G * nbp * cols);
    }
    DBuf<TC> scratch(c, (size_t)G * L + L);
    DBuf<double> f2;
    const double* fro2 = fn.p;
    if (!fro2) {
        f2.alloc(c, 1);
        CUDA_CHECK(cudaMemsetAsync(f2.p, 0, sizeof(double), c->stream));
        const long long len = (long long)n * cols;
        const int fb = (int)std::min<long long>(2LL * c->nsm, std::max(1LL, (len + 255) / 256));
        k_frob2_strided<<<fb, 256, 0, c->stream>>>(n, cols, A.p, A.s0, A.s1, f2.p);
        LAUNCH_CHECK(c);
        fro2 = f2.p;
    }
    QRParams<TC> P;
    P.n = n; P.c = cols; P.k = k; P.nb = nb; P.nbp = nbp; P.L = L;
    P.A = A.p; P.rs = A.s0; P.cs = A.s1;
    P.R = R; P.ldr = ldr;
    P.gwork = gwork.p;
    P.part = scratch.p;
    P.sums = scratch.p + (size_t)G * L;
    P.bar = c->dbarrier;
    P.status = c->dstatus;
    P.fnorm = fn.p;
    P.fro2 = fro2;
    P.wait_limit = c->wait_limit;
    CUDA_CHECK(cudaMemsetAsync(c->dbarrier, 0, 2 * sizeof(unsigned), c->stream));
    CUDA_CHECK(cudaFuncSetAttribute(k_qr_r<TC, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    CUDA_CHECK(cudaFuncSetAttribute(k_qr_r<TC, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    // a grid that fits in one thread-block cluster synchronises with the hardware
    // cluster barrier (~10x cheaper than the grid barrier); larger grids are cooperative
    if (G > 1 && G <= max_cluster_ctas(c, (const void*)k_qr_r<TC, true>, 256, smem)) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(G);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = c->stream;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = G;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        CUDA_CHECK(cudaLaunchKernelEx(&cfg, k_qr_r<TC, true>, P));
    } else {
        void* args[] = {&P};
        CUDA_CHECK(cudaLaunchCooperativeKernel((void*)k_qr_r<TC, false>, dim3(G), dim3(256), args, smem, c->stream));
    }
    count_launch(c);
    return false;
}
}  // namespace

void qr_r(tt_ctx* c, int n, int cols, MatView A, double* R, int ldr) {
    TT_REQUIRE(n > 0 && cols > 0, "qr_r: empty matrix %d x %d", n, cols);
    if (c->fast) qr_r_launch<float>(c, n, cols, A, R, ldr, nullptr);
    else qr_r_launch<double>(c, n, cols, A, R, ldr, nullptr);
}

// ============================================================== Jacobi SVD
namespace {
// Rotation of the column pair (a, b) of a one-sided Jacobi sweep, by one warp.
// Dot products and norms run over rows [0, m); the rotation is applied to rows
// [0, mr), mr >= m (rows m..mr-1 accumulate V when the caller needs it).  The
// squared norms in dn are refreshed from the rotated columns in the same pass.
// Returns whether the pair was rotated.  kGlobal: W and dn live in global memory
// shared by several CTAs (reads bypass L1).
template <typename T, bool kGlobal>
__device__ __forceinline__ T jld(const T* p) {
    if constexpr (kGlobal) return __ldcg(p);
    else return *p;
}
// Rotation of the column pair with squared norms al, be and product ga that makes
// the pair orthogonal: t = tan(theta) = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) with
// zeta = (be - al) / (2 ga), evaluated as sign(zeta) |2 ga| / (|be - al| + sqrt((be -
// al)^2 + (2 ga)^2)) (one square root and one division), cs = 1 / sqrt(1 + t^2),
// sn = cs t.  Returns false (no rotation) when the pair is orthogonal to tol,
// ga^2 <= tol^2 al be, or a column is numerically zero.
template <typename T>
__device__ __forceinline__ bool jacobi_rotation(T al, T be, T ga, T tol, T tiny, T& cs, T& sn) {
    if (!(al > tiny && be > tiny && ga * ga > (tol * tol * al) * be)) return false;
    const T d = be - al, g2 = T(2) * ga;
    const T r = sqrt(d * d + g2 * g2);
    const T t = copysign(T(1), d) * copysign(T(1), g2) * fabs(g2) / (fabs(d) + r);
    cs = rsqrt(T(1) + t * t);
    sn = cs * t;
    return true;
}

template <typename T, bool kGlobal>
__device__ __forceinline__ bool jacobi_pair(T* ca, T* cb, int a, int b, int m, int mr, T* dn, T tol, T tiny,
                                            double& flops) {
    const int lane = threadIdx.x & 31;
    const T al = jld<T, kGlobal>(dn + a), be = jld<T, kGlobal>(dn + b);
    T ga = T(0);
    for (int i = lane; i < m; i += 32) ga = fma(jld<T, kGlobal>(ca + i), jld<T, kGlobal>(cb + i), ga);
    ga = warp_sum(ga);
    flops += 2.0 * m;
    T cs, sn;
    if (!jacobi_rotation(al, be, ga, tol, tiny, cs, sn)) return false;
    T na = T(0), nb = T(0);
    for (int i = lane; i < mr; i += 32) {
        const T x = jld<T, kGlobal>(ca + i), y = jld<T, kGlobal>(cb + i);
        const T xn = cs * x - sn * y, yn = sn * x + cs * y;
        ca[i] = xn;
        cb[i] = yn;
        if (i < m) {
            na = fma(xn, xn, na);
            nb = fma(yn, yn, nb);
        }
    }
    na = warp_sum(na);
    nb = warp_sum(nb);
    if (lane == 0) {
        dn[a] = na;
        dn[b] = nb;
    }
    flops += 6.0 * mr + 4.0 * m;
    return true;
}

// Same rotation for m <= 32 KV rows (and no extra rows), with each lane's share of
// both columns held in registers between the dot product and the rotation, so the
// pair is read from L2 once.  The arithmetic and its order are those of
// jacobi_pair (rows past m contribute exact zeros).
template <typename T, int KV>
__device__ __forceinline__ bool jacobi_pair_reg(T* ca, T* cb, int a, int b, int m, T* dn, T tol, T tiny,
                                                double& flops) {
    const int lane = threadIdx.x & 31;
    const T al = __ldcg(dn + a), be = __ldcg(dn + b);
    T xa[KV], xb[KV];
#pragma unroll
    for (int k = 0; k < KV; ++k) {
        const int i = lane + 32 * k;
        xa[k] = i < m ? __ldcg(ca + i) : T(0);
        xb[k] = i < m ? __ldcg(cb + i) : T(0);
    }
    T ga = T(0);
#pragma unroll
    for (int k = 0; k < KV; ++k)
        if (lane + 32 * k < m) ga = fma(xa[k], xb[k], ga);
    ga = warp_sum(ga);
    flops += 2.0 * m;
    T cs, sn;
    if (!jacobi_rotation(al, be, ga, tol, tiny, cs, sn)) return false;
    T na = T(0), nb = T(0);
#pragma unroll
    for (int k = 0; k < KV; ++k) {
        const int i = lane + 32 * k;
        if (i < m) {
            const T xn = cs * xa[k] - sn * xb[k], yn = sn * xa[k] + cs * xb[k];
            ca[i] = xn;
            cb[i] = yn;
            na = fma(xn, xn, na);
            nb = fma(yn, yn, nb);
        }
    }
    na = warp_sum(na);
    nb = warp_sum(nb);
    if (lane == 0) {
        dn[a] = na;
        dn[b] = nb;
    }
    flops += 10.0 * m;
    return true;
}

// Round-robin (circle) pairing: round r pairs (r, npad-1) and ((r+p) mod (npad-1),
// (r-p) mod (npad-1)) for p = 1 .. npad/2-1; a column index >= n is a dummy.
__device__ __forceinline__ void circle_pair(int r, int p, int NR, int& a, int& b) {
    if (p == 0) { a = r; b = NR; } else { a = (r + p) % NR; b = (r - p + NR) % NR; }
}

// Sweeps over the whole grid: one warp per pair, a grid-wide barrier per round (the
// cluster barrier when the grid is one cluster, else the cooperative grid barrier).
// Columns with squared norm <= tiny_rel * frob2 are numerically zero and not rotated.
template <typename T, bool kCluster>
__global__ void __launch_bounds__(128)
k_jacobi(int m, int mr, int n, int npad, T* W, int ldw, int* flags, int max_sweeps, T tol, double tiny_rel,
         unsigned* bar, int* status, int* sweeps_used, const double* frob2, T* dn, double* flop_counter,
         long long wait_limit) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double myflops = 0.0;   // flops this warp performs (exact algorithmic count)
    const int gw = blockIdx.x * nw + warp, TW = gridDim.x * nw;
    const int P = npad / 2, NR = npad - 1;
    const T tiny = T(tiny_rel * __ldcg(frob2));
    int sw = 0;
    for (; sw < max_sweeps; ++sw) {
        int any = 0;
        for (int col = gw; col < n; col += TW) {
            const T* cc = W + (size_t)col * ldw;
            T s = T(0);
            for (int i = lane; i < m; i += 32) {
                const T x = __ldcg(cc + i);
                s = fma(x, x, s);
            }
            s = warp_sum(s);
            if (lane == 0) dn[col] = s;
            myflops += 2.0 * m;
        }
        group_barrier<kCluster>(bar, gridDim.x, status, wait_limit);
        for (int r = 0; r < NR; ++r) {
            for (int p = gw; p < P; p += TW) {
                int a, b;
                circle_pair(r, p, NR, a, b);
                if (a >= n || b >= n) continue;
                T* ca = W + (size_t)a * ldw;
                T* cb = W + (size_t)b * ldw;
                bool rot;
                if (mr == m && m <= 128) rot = jacobi_pair_reg<T, 4>(ca, cb, a, b, m, dn, tol, tiny, myflops);
                else if (mr == m && m <= 256) rot = jacobi_pair_reg<T, 8>(ca, cb, a, b, m, dn, tol, tiny, myflops);
                else rot = jacobi_pair<T, true>(ca, cb, a, b, m, mr, dn, tol, tiny, myflops);
                if (rot) any = 1;
            }
            group_barrier<kCluster>(bar, gridDim.x, status, wait_limit);
        }
        if (any && lane == 0) flags[sw] = 1;
        group_barrier<kCluster>(bar, gridDim.x, status, wait_limit);
        if (__ldcg(flags + sw) == 0) break;
        if (*(volatile int*)status == DEV_TIMEOUT) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps_used = sw;
    if (lane == 0 && flop_counter) atomicAdd(flop_counter, myflops);
}


// Sum over the L lanes of a lane group (L a power of two, groups aligned to L).
__device__ __forceinline__ double group_sum(double v, int L) {
    for (int o = L >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The rotation of jacobi_rotation with its angle taken in FP32 and its cosine in FP64.
// Only the transformation has to be orthogonal to FP64 precision, not the angle exact:
// t = tan theta = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (be - al) / (2 ga), is
// evaluated in FP32 on be - al and 2 ga scaled by the same power of two (exact), then
// cs = 1 / sqrt(1 + t^2) and sn = cs t in FP64 from that t, so cs^2 + sn^2 = 1 to FP64
// rounding and the rotation changes no singular value.  An angle off by FP32 rounding
// leaves |ga| at ~1e-7 of its value, which the next sweep removes.  The FP64
// dependency chain of a round shrinks from the ~35 operations of two FP64 square roots
// and a division to ~12.  Every lane of a group computes it from group-uniform al, be,
// ga; tg = t ga is the squared norm the rotation moves from column a to column b.
__device__ __forceinline__ bool ring_rotation(double al, double be, double ga, double tol, double tiny,
                                              double& cs, double& sn, double& tg) {
    const bool rot = al > tiny && be > tiny && ga * ga > (tol * tol * al) * be;
    cs = 1.0;
    sn = 0.0;
    tg = 0.0;
    if (rot) {
        const double d = be - al, g2 = 2.0 * ga;
        // power of two 2^-e with max(|d|, |g2|) 2^-e in [1, 2): both fit FP32 (|g2| >= 1e-28
        // |d| here, since columns below tiny are not rotated)
        const int hi = max(__double2hiint(fabs(d)), __double2hiint(fabs(g2)));
        const int e = ((hi >> 20) & 0x7ff) - 1023;
        const double sc = __hiloint2double((1023 - e) << 20, 0);
        const float z = (float)(d * sc) / (float)(g2 * sc);
        const float az = fabsf(z);
        const float r = az > 1e18f ? az : sqrtf(fmaf(az, az, 1.0f));
        const double t = (double)copysignf(1.0f / (az + r), z);
        cs = rsqrt(fma(t, t, 1.0));
        sn = cs * t;
        tg = t * ga;
    }
    return rot;
}

// One-sided Jacobi on one thread-block cluster with the columns held in distributed
// shared memory.  A slot holds the two columns of one pair of the current round of
// the circle ordering and is served by a group of L lanes (L = 4 .. 32, a warp serves
// 32 / L slots), each lane holding KV entries of both columns in registers: FP64
// issue, not the lane count, sets the speed of a round, and a group of L lanes
// spends the rotation's scalar work once for 32 / L pairs.  After rotating, a slot
// writes its columns straight into the slots that pair them in the next round (a
// ring shift: slot p's first column goes to slot p-1, its second to slot p+1, at the
// ends to slot 1's second and to slot P-1's own first; slot 0's second column is the
// fixed one), in another CTA's shared memory when the neighbour slot lives there.
// Every column carries its squared norm and its index, so a round reads only local
// shared memory and ends with one hardware cluster barrier; after each sweep the
// columns are back in their starting slots.  Squared norms are recomputed exactly at
// the start of each sweep and updated by the rotation in between (al - t ga, be +
// t ga), with an exact recompute when a column loses more than 3/4 of its squared
// norm.  Same ordering and stopping rule as k_jacobi.
template <int KV>
__global__ void __launch_bounds__(256)
k_jacobi_ring(int m, int n, int P, int L, int S, double* __restrict__ W, int ldw, int* __restrict__ flags,
              int max_sweeps, double tol, double tiny_rel, const double* __restrict__ frob2,
              int* __restrict__ sweeps_used) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) double rsm[];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int spw = 32 / L;
    const int gl = lane % L;                       // lane within the slot's group
    const int j = w * spw + lane / L;              // slot within this CTA
    const int blk = (int)cl.block_rank();
    const int p = blk * S + j;                     // slot within the cluster
    const bool live = j < S && p < P;
    const int NR = 2 * P - 1;
    // [buf][slot][col][m] data, [buf][slot][col] norms, [buf][slot][col] indices
    double* data = rsm;
    double* nrm = data + (size_t)4 * S * m;
    int* idx = reinterpret_cast<int*>(nrm + 4 * S);
    auto D = [&](int buf, int slot, int col) { return data + (((size_t)buf * S + slot) * 2 + col) * m; };
    auto NI = [&](int buf, int slot, int col) { return ((buf * S + slot) * 2 + col); };
    const double tiny = tiny_rel * *frob2;
    // this slot's columns in both buffers, and where they go in the next round (fixed
    // for the whole kernel: the ring shift does not depend on the round), resolved once
    // (scalars, not arrays, so that they stay in registers)
    const double *la0 = nullptr, *la1 = nullptr, *lb0 = nullptr, *lb1 = nullptr;
    double *ra0 = nullptr, *ra1 = nullptr, *rb0 = nullptr, *rb1 = nullptr;
    double *rna0 = nullptr, *rna1 = nullptr, *rnb0 = nullptr, *rnb1 = nullptr;
    int *ria0 = nullptr, *ria1 = nullptr, *rib0 = nullptr, *rib1 = nullptr;
    int lna = 0, lnb = 0;
    if (live) {
        int sa, ca, sb, cb;
        if (p == 0) { sa = 1; ca = 1; sb = 0; cb = 1; }
        else if (p == P - 1) { sa = p - 1; ca = 0; sb = p; cb = 0; }
        else { sa = p - 1; ca = 0; sb = p + 1; cb = 1; }
        la0 = D(0, j, 0); la1 = D(1, j, 0);
        lb0 = D(0, j, 1); lb1 = D(1, j, 1);
        ra0 = cl.map_shared_rank(D(0, sa % S, ca), sa / S);
        ra1 = cl.map_shared_rank(D(1, sa % S, ca), sa / S);
        rb0 = cl.map_shared_rank(D(0, sb % S, cb), sb / S);
        rb1 = cl.map_shared_rank(D(1, sb % S, cb), sb / S);
        rna0 = cl.map_shared_rank(nrm + NI(0, sa % S, ca), sa / S);
        rna1 = cl.map_shared_rank(nrm + NI(1, sa % S, ca), sa / S);
        rnb0 = cl.map_shared_rank(nrm + NI(0, sb % S, cb), sb / S);
        rnb1 = cl.map_shared_rank(nrm + NI(1, sb % S, cb), sb / S);
        ria0 = cl.map_shared_rank(idx + NI(0, sa % S, ca), sa / S);
        ria1 = cl.map_shared_rank(idx + NI(1, sa % S, ca), sa / S);
        rib0 = cl.map_shared_rank(idx + NI(0, sb % S, cb), sb / S);
        rib1 = cl.map_shared_rank(idx + NI(1, sb % S, cb), sb / S);
        lna = NI(0, j, 0);
        lnb = NI(0, j, 1);
        const int cols[2] = {p, p == 0 ? NR : NR - p};
        for (int c2 = 0; c2 < 2; ++c2) {
            const int ci = cols[c2];
            double* d = D(0, j, c2);
            for (int i = gl; i < m; i += L) d[i] = ci < n ? W[(size_t)ci * ldw + i] : 0.0;
            if (gl == 0) idx[NI(0, j, c2)] = ci;
        }
    }
    const int bstride = 2 * S;                     // norm/index entries per buffer
    cl.sync();
    int cur = 0, sw = 0;
    for (; sw < max_sweeps; ++sw) {
        int any = 0;
        for (int r = 0; r < NR; ++r) {
            const int nxt = cur ^ 1;
            double al = 0.0, be = 0.0;
            int ia = n, ib = n;
            double xa[KV], xb[KV];
            if (live) {
                const double* da = cur ? la1 : la0;
                const double* db = cur ? lb1 : lb0;
                al = nrm[lna + cur * bstride];
                be = nrm[lnb + cur * bstride];
                ia = idx[lna + cur * bstride];
                ib = idx[lnb + cur * bstride];
#pragma unroll
                for (int k = 0; k < KV; ++k) {
                    const int i = gl + L * k;
                    xa[k] = i < m ? da[i] : 0.0;
                    xb[k] = i < m ? db[i] : 0.0;
                }
            } else {
#pragma unroll
                for (int k = 0; k < KV; ++k) xa[k] = xb[k] = 0.0;
            }
            if (r == 0) {
                double na[2] = {0.0, 0.0}, nb[2] = {0.0, 0.0};
#pragma unroll
                for (int k = 0; k < KV; ++k) {
                    na[k & 1] = fma(xa[k], xa[k], na[k & 1]);
                    nb[k & 1] = fma(xb[k], xb[k], nb[k & 1]);
                }
                al = group_sum(na[0] + na[1], L);
                be = group_sum(nb[0] + nb[1], L);
            }
            double g[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int k = 0; k < KV; ++k) g[k & 3] = fma(xa[k], xb[k], g[k & 3]);
            const double ga = group_sum((g[0] + g[1]) + (g[2] + g[3]), L);
            // a slot that does not rotate (dummy column, no live slot, or orthogonal
            // already) applies the identity when another group of its warp rotates
            double cs = 1.0, sn = 0.0, tg = 0.0;
            const bool rot = live && ia < n && ib < n && ring_rotation(al, be, ga, tol, tiny, cs, sn, tg);
            if (rot) any = 1;
            if (__any_sync(FULL, rot)) {
#pragma unroll
                for (int k = 0; k < KV; ++k) {
                    const double xn = cs * xa[k] - sn * xb[k], yn = sn * xa[k] + cs * xb[k];
                    xa[k] = xn;
                    xb[k] = yn;
                }
                double an = al - tg, bn = be + tg;
                const bool refresh = rot && (an < 0.25 * al || bn < 0.25 * be);
                if (__any_sync(FULL, refresh)) {
                    double na = 0.0, nb = 0.0;
#pragma unroll
                    for (int k = 0; k < KV; ++k) {
                        na = fma(xa[k], xa[k], na);
                        nb = fma(xb[k], xb[k], nb);
                    }
                    na = group_sum(na, L);
                    nb = group_sum(nb, L);
                    if (refresh) {
                        an = na;
                        bn = nb;
                    }
                }
                if (rot) {
                    al = an;
                    be = bn;
                }
            }
            if (live) {
                double* pa = nxt ? ra1 : ra0;
                double* pb = nxt ? rb1 : rb0;
#pragma unroll
                for (int k = 0; k < KV; ++k) {
                    const int i = gl + L * k;
                    if (i < m) {
                        pa[i] = xa[k];
                        pb[i] = xb[k];
                    }
                }
                if (gl == 0) {
                    *(nxt ? rna1 : rna0) = al;
                    *(nxt ? ria1 : ria0) = ia;
                    *(nxt ? rnb1 : rnb0) = be;
                    *(nxt ? rib1 : rib0) = ib;
                }
            }
            cl.sync();
            cur = nxt;
        }
        if (any && gl == 0) flags[sw] = 1;
        cl.sync();
        if (__ldcg(flags + sw) == 0) break;
    }
    if (live) {
        for (int c2 = 0; c2 < 2; ++c2) {
            const int ci = idx[NI(cur, j, c2)];
            if (ci >= n) continue;
            const double* d = D(cur, j, c2);
            for (int i = gl; i < m; i += L) W[(size_t)ci * ldw + i] = d[i];
        }
    }
    if (blk == 0 && threadIdx.x == 0) *sweeps_used = sw;
}

// One-sided Jacobi of a small m x n matrix held entirely in the shared memory of one
// CTA: one warp per column pair of a round, block barriers between rounds, the same
// round-robin order, rotation and stopping rule as k_jacobi.  For matrices this small
// one SM's FP64 pipe finishes a round faster than a cross-CTA barrier completes.
__global__ void __launch_bounds__(1024)
k_jacobi_cta(int m, int n, int npad, double* __restrict__ W, int ldw, int max_sweeps, double tol, double tiny_rel,
             const double* __restrict__ frob2, int* __restrict__ sweeps_used, double* __restrict__ flop_counter) {
    extern __shared__ __align__(16) double jsm[];
    double* Ws = jsm;                              // n columns of m
    double* dn = Ws + (size_t)n * m;               // squared column norms
    int* flag = reinterpret_cast<int*>(dn + npad);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    for (int e = tid; e < n * m; e += blockDim.x) Ws[e] = W[(size_t)(e / m) * ldw + e % m];
    if (tid == 0) *flag = 0;
    const double tiny = tiny_rel * *frob2;
    const int P = npad / 2, NR = npad - 1;
    double myflops = 0.0;
    __syncthreads();
    int sw = 0;
    for (; sw < max_sweeps; ++sw) {
        for (int col = warp; col < n; col += nw) {
            const double* cc = Ws + (size_t)col * m;
            double a = 0.0;
            for (int i = lane; i < m; i += 32) a = fma(cc[i], cc[i], a);
            a = warp_sum(a);
            if (lane == 0) dn[col] = a;
            myflops += 2.0 * m;
        }
        __syncthreads();
        for (int r = 0; r < NR; ++r) {
            for (int p = warp; p < P; p += nw) {
                int a, b;
                circle_pair(r, p, NR, a, b);
                if (a >= n || b >= n) continue;
                if (jacobi_pair<double, false>(Ws + (size_t)a * m, Ws + (size_t)b * m, a, b, m, m, dn, tol, tiny,
                                               myflops) && lane == 0)
                    *flag = 1;
            }
            __syncthreads();
        }
        const int any = *(volatile int*)flag;
        __syncthreads();
        if (tid == 0) *flag = 0;
        if (!any) break;
    }
    for (int e = tid; e < n * m; e += blockDim.x) W[(size_t)(e / m) * ldw + e % m] = Ws[e];
    if (tid == 0) *sweeps_used = sw;
    if (lane == 0 && flop_counter) atomicAdd(flop_counter, myflops);
}

__global__ void k_frob2(long long len, const double* __restrict__ W, double* __restrict__ out) {
    double s = 0.0;
    for (long long i = threadIdx.x; i < len; i += blockDim.x) s = fma(W[i], W[i], s);
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

__global__ void k_colnorms(int m, int n, const double* __restrict__ W, int ldw, double* __restrict__ nrm) {
    const int col = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double x = W[(size_t)col * ldw + i];
        s = fma(x, x, s);
    }
    __shared__ double red[32];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        s = warp_sum(s);
        if (threadIdx.x == 0) nrm[col] = sqrt(s);
    }
}

// rank[i] = position of column i in descending order (ties by index)
__global__ void k_rank(int n, const double* __restrict__ nrm, int* __restrict__ rank) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = nrm[i];
        int r = 0;
        for (int j = 0; j < n; ++j) {
            const double w = nrm[j];
            r += (w > v) || (w == v && j < i);
        }
        rank[i] = r;
    }
}

// Columns the Jacobi sweep treats as numerically zero (squared norm <= 1e-30 ||A||_F^2,
// never rotated) get a zero left vector: normalising them would produce unit
// vectors that are not orthogonal to the others.
__global__ void k_permute_normalise(int m, int n, const double* __restrict__ W, int ldw,
                                    const double* __restrict__ nrm, const int* __restrict__ rank,
                                    double* __restrict__ sig, double* __restrict__ U,
                                    const double* __restrict__ frob2, const int* __restrict__ rowperm) {
    const int col = blockIdx.x;
    const int dst = rank[col];
    const double s = nrm[col];
    const double inv = (s > 0.0 && s * s > 1e-30 * *frob2) ? 1.0 / s : 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
        U[(size_t)dst * m + (rowperm ? rowperm[i] : i)] = W[(size_t)col * ldw + i] * inv;
    if (threadIdx.x == 0) sig[dst] = s;
}
}  // namespace

// Which Jacobi kernel: the cluster ring (columns in distributed shared memory, pairs
// spread over up to 16 SMs) for up to kJacobiRingMaxEntries entries; else the one-CTA
// shared-memory kernel for tiny matrices (or when no cluster can be formed); else the
// grid kernel with the columns in global memory.  GB300 issues a warp's FP64
// instruction over 16 cycles of an SM's FP64 pipe and a round is a chain of dependent
// instructions, so a round is bound by the longer of one warp's chain and the SM's FP64
// pipe: pairs are spread over as many SMs as a cluster has, a few warps to an SM.
constexpr long long kJacobiCtaMaxEntries = 4096;
constexpr long long kJacobiRingMaxEntries = 96 * 1024;

template <typename T>
static void jacobi_grid(tt_ctx* c, int m, int mr, int n, T* W, int ldw, T tol, double tiny_rel,
                        const double* frob2, int max_sweeps, double* fc, const char* tag) {
    const int npad = n + (n & 1);
    if constexpr (sizeof(T) == sizeof(double)) {
        const int P = npad / 2;
        // one cluster of at most 16 SMs: its FP64 pipes carry a round of (n/2) pairs x 12 m
        // flops; past about 1e5 entries a grid over more SMs (with its slower barrier)
        // finishes a round sooner
        if (mr == m && m <= 512 && P >= 2 && P <= 256 && (long long)m * n <= kJacobiRingMaxEntries) {
            // one cluster, columns in distributed shared memory.  Pick the slot width L
            // (lanes per pair) and entries per lane KV (L KV >= m) for the shortest round:
            // a round is bound either by one warp's instruction stream (~200 + 45 KV + 8
            // log2 L dependent instructions at ~8 cycles each: ncu shows "wait" stalls
            // dominating a one-warp-per-SM ring) or by the SM's FP64 pipe (warps per CTA x
            // (5 KV + log2 L + 12) FP64 instructions at 16 cycles each), over clusters of 16
            // or 8 CTAs.
            using RingKernel = void (*)(int, int, int, int, int, double*, int, int*, int, double, double,
                                        const double*, int*);
            const RingKernel kerns[5] = {k_jacobi_ring<2>, k_jacobi_ring<4>, k_jacobi_ring<8>, k_jacobi_ring<16>,
                                         k_jacobi_ring<32>};
            const int kvs[5] = {2, 4, 8, 16, 32};
            RingKernel kern = nullptr;
            int G = 0, S = 0, L = 0, threads = 0;
            size_t smem = 0;
            // the choice depends only on (device, m, n): cached, so that repeated shapes
            // skip the search and its attribute and occupancy queries
            struct RingCfg { int v, G, S, L, threads; size_t smem; };
            static std::mutex cache_mu;
            static std::map<std::tuple<int, int, int>, RingCfg> cache;
            const auto key = std::make_tuple(c->device, m, n);
            bool cached = false;
            {
                std::lock_guard<std::mutex> lk(cache_mu);
                const auto it = cache.find(key);
                if (it != cache.end()) {
                    const RingCfg& r = it->second;
                    kern = r.v >= 0 ? kerns[r.v] : nullptr;
                    G = r.G; S = r.S; L = r.L; threads = r.threads; smem = r.smem;
                    cached = true;
                }
            }
            double best = 1e30;
            int vbest = -1;
            for (int v = 0; v < 5 && !cached; ++v) {
                for (int l : {4, 8, 16, 32}) {
                    if (l * kvs[v] < m || (kvs[v] > 2 && l * kvs[v] >= 2 * m)) continue;
                    int lg = 0;
                    while ((1 << lg) < l) ++lg;
                    for (int g : {16, 8}) {
                        const int s = ceil_div(P, g);
                        const int warps = ceil_div(s, 32 / l);
                        if (warps > 8) continue;
                        const size_t sm = (size_t)4 * s * m * sizeof(double) + (size_t)4 * s * (sizeof(double) + sizeof(int));
                        if (sm > 200 * 1024) continue;
                        const int gg = ceil_div(P, s);
                        if (gg < 2) continue;
                        const double chain = 8.0 * (200.0 + 45.0 * kvs[v] + 8.0 * lg);
                        const double pipe = 16.0 * warps * (5.0 * kvs[v] + lg + 12.0);
                        const double cost = std::max(chain, pipe);
                        if (cost >= best) continue;
                        CUDA_CHECK(cudaFuncSetAttribute(kerns[v], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        227 * 1024));
                        if (max_cluster_ctas(c, (const void*)kerns[v], 32 * warps, sm) < gg) continue;
                        best = cost;
                        kern = kerns[v];
                        vbest = v;
                        G = gg;
                        S = s;
                        L = l;
                        threads = 32 * warps;
                        smem = sm;
                    }
                }
            }
            if (!cached) {
                std::lock_guard<std::mutex> lk(cache_mu);
                cache[key] = RingCfg{G >= 2 ? vbest : -1, G, S, L, threads, smem};
            }
            if (G >= 2 && kern) {
                DBuf<int> flags(c, max_sweeps + 1);
                CUDA_CHECK(cudaMemsetAsync(flags.p, 0, (max_sweeps + 1) * sizeof(int), c->stream));
                int* sweeps = flags.p + max_sweeps;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(G);
                cfg.blockDim = dim3(threads);
                cfg.dynamicSmemBytes = smem;
                cfg.stream = c->stream;
                cudaLaunchAttribute attr;
                attr.id = cudaLaunchAttributeClusterDimension;
                attr.val.clusterDim.x = G;
                attr.val.clusterDim.y = 1;
                attr.val.clusterDim.z = 1;
                cfg.attrs = &attr;
                cfg.numAttrs = 1;
                CUDA_CHECK(cudaLaunchKernelEx(&cfg, kern, m, n, P, L, S, (double*)W, ldw, flags.p, max_sweeps,
                                              (double)tol, tiny_rel, frob2, sweeps));
                count_launch(c);
                static const bool log = getenv("TT_LOG_ROUND") != nullptr;
                if (log) {
                    int h = 0;
                    read_back(c, (const int*)sweeps, &h, 1);
                    fprintf(stderr, "jacobi%s-ring m=%d n=%d ctas=%d L=%d slots=%d sweeps=%d\n", tag, m, n, G, L, S, h);
                }
                return;
            }
        }
    }
    if constexpr (sizeof(T) == sizeof(double)) {
        if ((long long)m * n <= kJacobiCtaMaxEntries && mr == m) {
            // small matrix: one CTA, everything in shared memory
            DBuf<int> sw(c, 1);
            const int threads = 32 * std::min(32, std::max(1, npad / 2));
            const size_t smem = ((size_t)n * m + npad) * sizeof(double) + 16;
            k_jacobi_cta<<<1, threads, smem, c->stream>>>(m, n, npad, (double*)W, ldw, max_sweeps, (double)tol,
                                                          tiny_rel, frob2, sw.p, fc);
            LAUNCH_CHECK(c);
            static const bool log = getenv("TT_LOG_ROUND") != nullptr;
            if (log) {
                int h = 0;
                read_back(c, (const int*)sw.p, &h, 1);
                fprintf(stderr, "jacobi%s-cta m=%d n=%d sweeps=%d\n", tag, m, n, h);
            }
            return;
        }
    }
    const int wpb = 4;
    const int G = std::max(1, std::min(c->nsm, ceil_div(npad / 2, wpb)));
    DBuf<int> flags(c, max_sweeps + 1);
    CUDA_CHECK(cudaMemsetAsync(flags.p, 0, (max_sweeps + 1) * sizeof(int), c->stream));
    CUDA_CHECK(cudaMemsetAsync(c->dbarrier, 0, 2 * sizeof(unsigned), c->stream));
    DBuf<T> dn(c, n);
    int* sweeps = flags.p + max_sweeps;
    int mm = m, mmr = mr, nn = n, np_ = npad, ld = ldw, ms = max_sweeps;
    T tl = tol;
    double tr = tiny_rel;
    unsigned* bar = c->dbarrier;
    int* st = c->dstatus;
    int* fl = flags.p;
    const double* f2 = frob2;
    T* dnp = dn.p;
    long long wl = c->wait_limit;
    if (G > 1 && G <= max_cluster_ctas(c, (const void*)k_jacobi<T, true>, 32 * wpb, 0)) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(G);
        cfg.blockDim = dim3(32 * wpb);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = c->stream;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = G;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        CUDA_CHECK(cudaLaunchKernelEx(&cfg, k_jacobi<T, true>, mm, mmr, nn, np_, W, ld, fl, ms, tl, tr, bar, st,
                                      sweeps, f2, dnp, fc, wl));
    } else {
        void* args[] = {&mm, &mmr, &nn, &np_, &W, &ld, &fl, &ms, &tl, &tr, &bar, &st, &sweeps, &f2, &dnp, &fc, &wl};
        CUDA_CHECK(cudaLaunchCooperativeKernel((void*)k_jacobi<T, false>, dim3(G), dim3(32 * wpb), args, 0,
                                               c->stream));
    }
    count_launch(c);
    static const bool log = getenv("TT_LOG_ROUND") != nullptr;
    if (log) {
        int sw = 0;
        read_back(c, (const int*)sweeps, &sw, 1);
        fprintf(stderr, "jacobi%s m=%d n=%d sweeps=%d\n", tag, m, n, sw);
    }
}

static void jacobi_columns(tt_ctx* c, int m, int n, double* W, double* sig, double* U, double ortho_tol,
                           const int* rowperm) {
    // W: m x n column-major (ld m), overwritten by W V (orthogonal columns); row i of W
    // is row rowperm[i] of U (identity when null)
    const int max_sweeps = 60;
    // Orthogonality target: FP64 dot products of nearly orthogonal columns carry
    // rounding noise of order m eps_mach, so a tighter target only re-rotates noise.
    const double tol = std::max(ortho_tol, 4.0 * m * 2.220446049250313e-16);
    DBuf<double> frob2(c, 1);
    k_frob2<<<1, 256, 0, c->stream>>>((long long)m * n, W, frob2.p);
    LAUNCH_CHECK(c);
    if (n > 1) {
        // flops are counted on the device (dots, rotations and norm passes performed)
        // algorithmic work of the launch: the dense SVD count for singular values and
        // the m x n left singular vectors, 14 m n^2 + 8 n^3 (Golub and Van Loan, m >= n),
        // whatever number of sweeps the Jacobi iteration takes; bytes: W read and written
        const double dm = m, dn = n;
        ProfScope prof(c, PROF_JACOBI, 14.0 * dm * dn * dn + 8.0 * dn * dn * dn, 16.0 * dm * dn);
        jacobi_grid<double>(c, m, m, n, W, m, tol, 1e-30, frob2.p, max_sweeps, nullptr, "");
    }
    DBuf<double> nrm(c, n);
    DBuf<int> rank(c, n);
    k_colnorms<<<n, 256, 0, c->stream>>>(m, n, W, m, nrm.p);
    LAUNCH_CHECK(c);
    k_rank<<<ceil_div(n, 256), 256, 0, c->stream>>>(n, nrm.p, rank.p);
    LAUNCH_CHECK(c);
    k_permute_normalise<<<n, 256, 0, c->stream>>>(m, n, W, m, nrm.p, rank.p, sig, U, frob2.p, rowperm);
    LAUNCH_CHECK(c);
}

void left_svd(tt_ctx* c, int m, int n, MatView A, double* sig, double* U, double ortho_tol) {
    TT_REQUIRE(m > 0 && n > 0, "left_svd: empty matrix");
    // The SVD is FP64 on both precision paths.  A^T P = Q R (Householder with column
    // pivoting, R is k x m with k = min(m, n)) gives P^T A = R^T Q^T: the left singular
    // vectors of A are those of the m x k matrix R^T with rows permuted by P, and
    // one-sided Jacobi on R^T converges in far fewer sweeps than on A itself (the
    // triangular factor of a pivoted QR has nearly orthogonal, graded columns;
    // QR-preconditioned Jacobi, Drmac and Veselic 2008).
    PrecScope fp64(c, 0);
    const int k = std::min(m, n);
    DBuf<double> R(c, (size_t)k * m);
    DBuf<int> perm(c, m);
    const bool pivoted = qr_r_launch<double>(c, n, m, trans(A), R.p, m, perm.p);   // R: k x m row-major
    // W = R^T column-major (m x k): W(i, j) = R(j, i) at j*m + i = R[j*m + i]
    DBuf<double> W(c, (size_t)m * k);
    CUDA_CHECK(cudaMemcpyAsync(W.p, R.p, (size_t)m * k * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    jacobi_columns(c, m, k, W.p, sig, U, ortho_tol, pivoted ? perm.p : nullptr);
}

// ============================================================== truncation
namespace {
__global__ void k_trunc_first(const double* __restrict__ s, int p, double eps, int maxr, TruncInfo* info) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double tot = 0.0;
    for (int i = p - 1; i >= 0; --i) tot += s[i] * s[i];
    info->nrm = sqrt(tot);
    const double d2 = eps > 0.0 ? 0.5 * eps * eps * tot : 0.0;
    info->delta2 = d2;
    int r = p;
    if (eps > 0.0) {
        double tail = 0.0;
        r = p;
        for (int i = p - 1; i >= 1; --i) {
            tail += s[i] * s[i];
            if (tail <= d2) r = i; else break;
        }
    } else {
        r = 0;
        for (int i = 0; i < p; ++i) r += s[i] > 0.0;
    }
    if (r < 1) r = 1;
    info->capped = 0;
    if (maxr > 0 && r > maxr) {
        r = maxr;
        info->capped = 1;
    }
    info->r1 = r;
}
__global__ void k_trunc_second(const double* __restrict__ s, int p, double eps, int maxr, TruncInfo* info) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double d2 = info->delta2;
    int r = p;
    if (eps > 0.0) {
        double tail = 0.0;
        for (int i = p - 1; i >= 1; --i) {
            tail += s[i] * s[i];
            if (tail <= d2) r = i; else break;
        }
    } else {
        r = 0;
        for (int i = 0; i < p; ++i) r += s[i] > 0.0;
    }
    if (r < 1) r = 1;
    if (maxr > 0 && r > maxr) {
        r = maxr;
        info->capped |= 2;
    }
    info->r2 = r;
    double kept = 0.0;
    for (int i = r - 1; i >= 0; --i) kept += s[i] * s[i];
    info->nrm_after = sqrt(kept);
}
}  // namespace

void trunc_first(tt_ctx* c, const double* sig1, int p1, double eps, TruncInfo* dinfo, int maxr) {
    k_trunc_first<<<1, 32, 0, c->stream>>>(sig1, p1, eps, maxr, dinfo);
    LAUNCH_CHECK(c);
}
void trunc_second(tt_ctx* c, const double* sig2, int p2, double eps, TruncInfo* dinfo, int maxr) {
    k_trunc_second<<<1, 32, 0, c->stream>>>(sig2, p2, eps, maxr, dinfo);
    LAUNCH_CHECK(c);
}

}  // namespace tt
