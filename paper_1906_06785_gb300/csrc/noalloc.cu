// Allocation-free inner product of two trains (tt_dot_noalloc).
//
// Some callers cannot allocate device memory at the moment they need an inner
// product: a process that has handed its whole device memory to its own pool up
// front (so any further cudaMalloc fails), a latency-critical loop that must not
// enter an allocator at all, or code running while another component holds the
// allocator.  tt_dot_noalloc computes the same value as tt_dot with all of its
// scratch in one statically sized device array, so the call allocates nothing.
// The paper has no counterpart of this entry point.
#include <mutex>

#include "tt.cuh"

// Scratch of tt_dot_noalloc: 2^21 doubles (16 MiB) per device, held for the life
// of the process.  Nothing in it needs to start at zero: every intermediate is
// written in full before it is read.  Calls that overlap in time on one device
// share it and race.
static constexpr size_t kNoAllocDoubles = size_t(1) << 21;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

namespace tt {
namespace {

// Device address of the scratch array, resolved once per device with that device
// current, and cached.  (In host code the symbol is only a handle, never a device
// pointer.)
double* scratch_address(int device) {
    static std::mutex mu;
    static double* addr[64] = {nullptr};
    TT_REQUIRE(device >= 0 && device < 64, "device index %d out of range", device);
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        int cur = -1;
        CUDA_CHECK(cudaGetDevice(&cur));
        if (cur != device) CUDA_CHECK(cudaSetDevice(device));
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (cur != device) CUDA_CHECK(cudaSetDevice(cur));
        if (e != cudaSuccess)
            TT_THROW(TT_ECUDA, "cudaGetSymbolAddress of the allocation-free scratch: %s", cudaGetErrorString(e));
        addr[device] = static_cast<double*>(p);
    }
    return addr[device];
}

__global__ void k_frob_dot_out(int n, const double* __restrict__ a, const double* __restrict__ b,
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

// <a, b> by the same contractions as the library's dot (core 1, then core 2, with
// core 3 as a Gram matrix), every intermediate and every split-K partial placed in
// the static scratch.  Returns the value on the host.
double dot_noalloc(tt_ctx* c, const tt_t* a, const tt_t* b) {
    TT_REQUIRE(a->n_t == b->n_t && a->n_xi == b->n_xi && a->n_x == b->n_x, "dot: shape mismatch");
    PrecScope fp64(c, 0);
    const int n_t = a->n_t, n_xi = a->n_xi, n_x = a->n_x;
    const int ra1 = a->r1, ra2 = a->r2, rb1 = b->r1, rb2 = b->r2;
    const size_t nW1 = (size_t)ra1 * rb1, nT = (size_t)ra1 * n_xi * rb2, nW2 = (size_t)ra2 * rb2;
    const size_t fixed = nW1 + nT + 2 * nW2 + 1;
    if (fixed > kNoAllocDoubles)
        TT_THROW(TT_EINVAL,
                 "tt_dot_noalloc: ranks (%d,%d) and (%d,%d) with n_xi=%d need %zu scratch doubles; the "
                 "static scratch holds %zu",
                 ra1, ra2, rb1, rb2, n_xi, fixed, kNoAllocDoubles);
    double* s = scratch_address(c->device);
    double* W1 = s;
    double* T = W1 + nW1;
    double* W2 = T + nT;
    double* G3 = W2 + nW2;
    double* res = G3 + nW2;
    double* ws = res + 1;
    const size_t wsl = kNoAllocDoubles - fixed;
    gemm_ws(c, ra1, rb1, n_t, 1.0, trans(colmaj(a->z1, n_t)), colmaj(b->z1, n_t), 0.0, rowmaj(W1, rb1), ws, wsl);
    gemm_ws(c, ra1, n_xi * rb2, rb1, 1.0, rowmaj(W1, rb1), rowmaj(b->z2, (long long)n_xi * rb2), 0.0,
            rowmaj(T, (long long)n_xi * rb2), ws, wsl);
    gemm_ws(c, ra2, rb2, ra1 * n_xi, 1.0, trans(rowmaj(a->z2, ra2)), rowmaj(T, rb2), 0.0, rowmaj(W2, rb2), ws, wsl);
    gemm_ws(c, ra2, rb2, n_x, 1.0, trans(rowmaj(a->z3, ra2)), rowmaj(b->z3, rb2), 0.0, rowmaj(G3, rb2), ws, wsl);
    k_frob_dot_out<<<1, 256, 0, c->stream>>>(ra2 * rb2, W2, G3, res);
    LAUNCH_CHECK(c);
    double h = 0.0;
    read_back(c, (const double*)res, &h, 1);   // through the context's pinned staging buffer
    return h;
}

}  // namespace
}  // namespace tt

extern "C" int tt_dot_noalloc(tt_ctx* ctx, const tt_t* a, const tt_t* b, double* out) {
    try {
        TT_REQUIRE(ctx && a && b && out, "null argument");
        *out = tt::dot_noalloc(ctx, a, b);
        return TT_OK;
    } catch (const tt::Error& e) {
        if (ctx) ctx->err = e.what();
        return e.code;
    } catch (const std::exception& e) {
        if (ctx) ctx->err = e.what();
        return TT_ECUDA;
    }
}
