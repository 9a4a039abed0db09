// Shared host/device infrastructure of the GPU solver: context, errors,
// stream-ordered device buffers, launch accounting and the bounded grid-wide
// barrier used by the cooperative (persistent) kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/tt_stochns.h"

namespace tt {

// ---------------------------------------------------------------- errors
struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define TT_THROW(code, ...)                                      \
    do {                                                         \
        char _b[400];                                            \
        snprintf(_b, sizeof(_b), __VA_ARGS__);                   \
        throw ::tt::Error((code), std::string(_b));              \
    } while (0)

#define TT_REQUIRE(cond, ...)                                    \
    do {                                                         \
        if (!(cond)) TT_THROW(TT_EINVAL, __VA_ARGS__);           \
    } while (0)

#define CUDA_CHECK(expr)                                                              \
    do {                                                                              \
        cudaError_t _e = (expr);                                                      \
        if (_e != cudaSuccess)                                                        \
            TT_THROW(_e == cudaErrorMemoryAllocation ? TT_ENOMEM : TT_ECUDA,          \
                     "%s:%d %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(_e)); \
    } while (0)

// Device status word written by kernels whose waits are bounded.
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_NAN = 2 };

}  // namespace tt

// ---------------------------------------------------------------- profiling
// Opt-in per-kernel-class timing with CUDA events on the context stream, plus
// the algorithmic flops and bytes of every timed launch.
enum ProfSlot : int {
    PROF_QR = 0, PROF_JACOBI, PROF_GEMM, PROF_SPMM, PROF_BAND_SOLVE, PROF_BAND_FACTOR,
    PROF_CORE, PROF_ASSEMBLY, PROF_CONV, PROF_NSLOTS
};
struct ProfData {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[PROF_NSLOTS];
    std::vector<cudaEvent_t> pool;
    double ms[PROF_NSLOTS] = {0};
    double flops[PROF_NSLOTS] = {0};
    double bytes[PROF_NSLOTS] = {0};
    long long n[PROF_NSLOTS] = {0};
};

// ---------------------------------------------------------------- context
struct tt_ctx {
    bool prof = false;
    ProfData pd;
    // Compute precision of the SpMM, GEMM, Householder R factor and banded solves:
    // 0 = FP64, 1 = FP32 arithmetic on FP64-stored data (the mixed path).  SVDs
    // (with their R factors), inner products, Hessenberg solves and band
    // factorisations are FP64 always.
    int fast = 0;
    // Truncations inside GMRES take the randomized variant (round_rand) when set; the
    // sketches draw from a counter-based generator at seed rand_seq, advanced per call
    bool randomized = false;
    unsigned long long rand_seq = 0x243F6A8885A308D3ull;
    // Truncations with eps >= 5e-6 may take the Gram route (FP64 GEMMs and
    // eigenpairs of small Gram matrices instead of Householder R factors).
    bool gram_ok = true;
    cudaStream_t stream = nullptr;
    int device = 0;
    int nsm = 0;
    long long launches = 0;
    std::string err = "ok";
    // device memory: the caller's stream-ordered allocator when given, else the
    // library's own cudaMallocAsync pool
    tt_alloc_fn alloc_fn = nullptr;
    tt_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    // small pinned host buffer for scalar read-back
    void* pinned = nullptr;
    // device status word (bounded waits) + barrier counters
    int* dstatus = nullptr;
    unsigned* dbarrier = nullptr;   // [count, generation] per barrier slot
    // polls a block makes at a grid barrier before it gives up (DEV_TIMEOUT): seconds
    // with the back-off, far beyond any wait of a healthy launch
    long long wait_limit = 20000000LL;
    double* dprof_flops = nullptr;  // device-counted flops per profiling slot
    // second context on its own stream (created on first use) on which the pressure
    // train of a (velocity, pressure) pair is truncated while the velocity train is
    // truncated here: the two truncations are independent and each uses only a few SMs
    tt_ctx* side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace tt {

inline void count_launch(tt_ctx* c, int n = 1) { c->launches += n; }

// Device memory of the context: the caller's allocator when it gave one, else
// the stream-ordered pool.  Both are ordered on the context stream.
inline void* ctx_malloc(tt_ctx* c, size_t bytes) {
    if (!bytes) return nullptr;
    if (c->alloc_fn) {
        void* p = c->alloc_fn(bytes, (void*)c->stream, c->alloc_user);
        if (!p) TT_THROW(TT_ENOMEM, "caller allocator returned NULL for %zu bytes", bytes);
        return p;
    }
    void* p = nullptr;
    const cudaError_t e = cudaMallocAsync(&p, bytes, c->stream);
    if (e != cudaSuccess) TT_THROW(TT_ENOMEM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return p;
}
inline void ctx_free(tt_ctx* c, void* p, size_t bytes) {
    if (!p) return;
    if (c->free_fn) c->free_fn(p, bytes, (void*)c->stream, c->alloc_user);
    else if (!c->alloc_fn) cudaFreeAsync(p, c->stream);
}

#define LAUNCH_CHECK(ctx)                                                         \
    do {                                                                          \
        ::tt::count_launch(ctx);                                                  \
        cudaError_t _e = cudaGetLastError();                                      \
        if (_e != cudaSuccess)                                                    \
            TT_THROW(TT_ECUDA, "%s:%d launch: %s", __FILE__, __LINE__, cudaGetErrorString(_e)); \
    } while (0)

// Stream-ordered device buffer from the context's allocator (ctx_malloc).
template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    tt_ctx* c = nullptr;
    DBuf() = default;
    DBuf(tt_ctx* ctx, size_t count) { alloc(ctx, count); }
    void alloc(tt_ctx* ctx, size_t count) {
        release();
        c = ctx;
        n = count;
        p = static_cast<T*>(ctx_malloc(ctx, count * sizeof(T)));
    }
    void release() {
        if (p) ctx_free(c, p, n * sizeof(T));
        p = nullptr;
        n = 0;
    }
    ~DBuf() { release(); }
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), c(o.c) { o.p = nullptr; o.n = 0; }
    DBuf& operator=(DBuf&& o) noexcept {
        release();
        p = o.p; n = o.n; c = o.c;
        o.p = nullptr; o.n = 0;
        return *this;
    }
};

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Copy scalars device -> host through the pinned buffer (synchronises the stream).
template <typename T>
inline void read_back(tt_ctx* c, const T* dsrc, T* hdst, size_t n) {
    size_t bytes = n * sizeof(T);
    if (bytes > 4096) {
        CUDA_CHECK(cudaMemcpyAsync(hdst, dsrc, bytes, cudaMemcpyDeviceToHost, c->stream));
        CUDA_CHECK(cudaStreamSynchronize(c->stream));
        return;
    }
    CUDA_CHECK(cudaMemcpyAsync(c->pinned, dsrc, bytes, cudaMemcpyDeviceToHost, c->stream));
    CUDA_CHECK(cudaStreamSynchronize(c->stream));
    memcpy(hdst, c->pinned, bytes);
}

// Check the device status word after kernels with bounded waits.
void check_status(tt_ctx* c);

// The context's side context (see tt_ctx::side), created on first use.
tt_ctx* side_ctx(tt_ctx* c);
void destroy_side(tt_ctx* c);

// Records an event pair around the launches in its scope when profiling is on.
struct ProfScope {
    tt_ctx* c;
    int slot;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(tt_ctx* ctx, int s, double flops, double bytes);
    ~ProfScope();
};
void prof_resolve(tt_ctx* c);

// Sets whether GMRES truncations are randomized for its scope (restores on exit).
struct RandScope {
    tt_ctx* c;
    bool saved;
    RandScope(tt_ctx* ctx, bool on) : c(ctx), saved(ctx->randomized) { c->randomized = on; }
    ~RandScope() { c->randomized = saved; }
};

// Sets the context's compute precision for its scope (restores on exit).
struct PrecScope {
    tt_ctx* c;
    int saved;
    PrecScope(tt_ctx* ctx, int fast) : c(ctx), saved(ctx->fast) { c->fast = fast; }
    ~PrecScope() { c->fast = saved; }
};

}  // namespace tt

// ---------------------------------------------------------------- tensor train
// Device-resident train, layouts as in include/tt_stochns.h.
struct tt_t {
    tt_ctx* ctx = nullptr;
    int n_t = 0, n_xi = 0, n_x = 0, r1 = 0, r2 = 0;
    int cap1 = 0, cap2 = 0;   // rank capacities the allocation holds (>= r1, r2)
    size_t bytes = 0;         // size of the allocation at base
    double* base = nullptr;
    double* z1 = nullptr;   // [r1][n_t]
    double* z2 = nullptr;   // [r1][n_xi][r2]
    double* z3 = nullptr;   // [n_x][r2]
};

namespace tt {

// New train; cap1, cap2 <= 0 mean capacities equal to the ranks.
tt_t* tt_alloc(tt_ctx* c, int n_t, int n_xi, int n_x, int r1, int r2, int cap1 = 0, int cap2 = 0);
void tt_free(tt_t* t);
using TTPtr = std::unique_ptr<tt_t, void (*)(tt_t*)>;
inline TTPtr wrap(tt_t* t) { return TTPtr(t, tt_free); }

// ---------------------------------------------------------------- device helpers
#ifdef __CUDACC__
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Grid-wide barrier for cooperative launches.  bar[0] counts arrivals, bar[1] is
// the generation.  Every wait is bounded: after `limit` polls the block records
// DEV_TIMEOUT in *status and leaves; once DEV_TIMEOUT is set, later barriers return
// at once, so a kernel that lost a block still terminates.  Other status values
// (a non-finite pivot met by an earlier kernel) do not affect the barrier.
__device__ __forceinline__ void grid_barrier(unsigned* bar, unsigned nblocks, int* status, long long limit) {
    __syncthreads();
    if (nblocks == 1) return;   // a one-block launch needs only the block barrier
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = bar + 1;
        unsigned gen = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long polls = 0;
            while (*vgen == gen) {
                if (*(volatile int*)status == DEV_TIMEOUT) break;
                if (++polls > limit) {
                    atomicExch(status, DEV_TIMEOUT);
                    break;
                }
                if (polls > 64) __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Barrier across all CTAs of a launch.  kCluster: the launch is one thread-block
// cluster and the hardware cluster barrier (release/acquire at cluster scope, which
// orders the CTAs' global and shared memory accesses) replaces the software grid
// barrier; every CTA of a cluster is resident by construction, so it cannot wait
// on an absent CTA.
template <bool kCluster>
__device__ __forceinline__ void group_barrier(unsigned* bar, unsigned nblocks, int* status, long long limit) {
    if constexpr (kCluster) {
        __syncthreads();
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    } else {
        grid_barrier(bar, nblocks, status, limit);
    }
}
#endif

// Largest single-cluster grid (CTAs) that can run `kernel` with `threads` threads and
// `smem` bytes of dynamic shared memory per CTA on this device: 16 when the
// non-portable size is schedulable, else 8, else 0 (no cluster launch).
int max_cluster_ctas(tt_ctx* c, const void* kernel, int threads, size_t smem);

}  // namespace tt
