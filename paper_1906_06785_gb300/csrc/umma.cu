// 3x3 convolutions of the learned mean-Oseen solve on the 5th-generation tensor
// cores (tcgen05): an implicit GEMM D[pixel, o] = sum_k A[pixel, k] B[o, k] with
// k = (input channel, tap), A gathered from the FP32 activations on the fly (the
// im2col matrix is never stored) and rounded to BF16, B the BF16 weights, D in
// FP32 in tensor memory.  One CTA owns 128 output pixels x Cout (<= 256) channels:
// its four warps stage K-chunks of A and B in shared memory in the canonical
// no-swizzle K-major layout (8-row x 16-byte core matrices), one thread issues the
// tcgen05.mma instructions (M = 128, N = Cout, K = 16 each) and commits them to an
// mbarrier, and the staging of the next chunk overlaps the MMAs of the current one
// (two buffers).  The epilogue reads the accumulator rows back with tcgen05.ld
// (warp w owns TMEM lanes 32w..32w+31 = pixels), adds the bias, applies the ReLU
// or the backward gate and stores pixel-contiguous rows.
#include <cuda_bf16.h>

#include <cstdint>

#include "umma.cuh"

namespace tt {
namespace {

constexpr int UM = 128;            // pixels per CTA (MMA M)
constexpr int UK = 64;             // K elements per staged chunk
constexpr int A_BYTES = UM * UK * 2;
constexpr uint32_t kCoreBytes = 128;             // 8 rows x 16 bytes
constexpr uint32_t kLBO = kCoreBytes;            // next core matrix along K
constexpr uint32_t kSBO = (UK / 8) * kCoreBytes; // next 8-row group

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of tcgen05 for a no-swizzle K-major operand:
// start address, leading-dimension byte offset (between core matrices along K),
// stride-dimension byte offset (between 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16 A and B,
// both K-major, N >> 3 and M >> 4.
__device__ __forceinline__ uint32_t instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (row, k) of a staged tile in the canonical layout
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
    return (uint32_t)(row >> 3) * kSBO + (uint32_t)(k >> 3) * kLBO + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Wait for the completion of the phase with the given parity; bounded.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_addr(bar);
    for (long long it = 0; it < (1LL << 26); ++it) {
        uint32_t done = 0;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// out[b][o][p] = act(bias[o] + sum_{c, tap} W[o][c][tap] X[b][c][p + tap offset]) for
// the B images of the FP32 activations X[b][c][p] (zero padding), BF16 operands,
// FP32 accumulation; with a gate, out *= (gate > 0); with zout the pre-activation
// is stored too.  Requires Cout % 16 == 0, Cout <= 256.
__global__ void __launch_bounds__(128)
k_conv3x3_umma(int B, int Cin, int Cout, int nx, int ny, const float* __restrict__ X,
               const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias, int relu,
               const float* __restrict__ gate, float* __restrict__ zout, float* __restrict__ out,
               int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char usm[];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int npix = nx * ny;
    const long long rows = (long long)B * npix;
    const long long g0 = (long long)blockIdx.x * UM;
    const int K = Cin * 9, nK = (K + UK - 1) / UK;
    const int B_BYTES = Cout * UK * 2;
    unsigned char* Abuf = usm;                                 // [2][A_BYTES]
    unsigned char* Bbuf = usm + 2 * A_BYTES;                   // [2][B_BYTES]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(Bbuf + 2 * B_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
    const uint32_t ncols = Cout <= 32 ? 32u : Cout <= 64 ? 64u : Cout <= 128 ? 128u : 256u;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = instr_desc(UM, Cout);

    // this thread's pixel
    const long long g = g0 + tid;
    const bool valid = g < rows;
    const int b = valid ? (int)(g / npix) : 0;
    const int p = valid ? (int)(g % npix) : 0;
    const int py = p / nx, px = p % nx;
    const float* xb = X + (size_t)b * Cin * npix;

    bool ok = true;
    for (int kc = 0; kc < nK; ++kc) {
        const int buf = kc & 1;
        if (kc >= 2 && !mbar_wait(&mbar[buf], (uint32_t)(((kc - 2) >> 1) & 1))) { ok = false; break; }
        unsigned char* A = Abuf + buf * A_BYTES;
        unsigned char* Bt = Bbuf + buf * B_BYTES;
        // A: row tid, 8 groups of 8 consecutive k
        for (int grp = 0; grp < UK / 8; ++grp) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = kc * UK + grp * 8 + e;
                float x = 0.0f;
                if (valid && k < K) {
                    const int c = k / 9, t = k - 9 * c;
                    const int yy = py + t / 3 - 1, xx = px + t % 3 - 1;
                    if (yy >= 0 && yy < ny && xx >= 0 && xx < nx) x = xb[(size_t)c * npix + yy * nx + xx];
                }
                v[e] = x;
            }
            __nv_bfloat162 h0 = __floats2bfloat162_rn(v[0], v[1]), h1 = __floats2bfloat162_rn(v[2], v[3]);
            __nv_bfloat162 h2 = __floats2bfloat162_rn(v[4], v[5]), h3 = __floats2bfloat162_rn(v[6], v[7]);
            uint4 q;
            q.x = *reinterpret_cast<uint32_t*>(&h0);
            q.y = *reinterpret_cast<uint32_t*>(&h1);
            q.z = *reinterpret_cast<uint32_t*>(&h2);
            q.w = *reinterpret_cast<uint32_t*>(&h3);
            *reinterpret_cast<uint4*>(A + tile_off(tid, grp * 8)) = q;
        }
        // B: Cout rows x 8 groups of 8 k
        for (int e = tid; e < Cout * (UK / 8); e += UM) {
            const int o = e / (UK / 8), grp = e % (UK / 8);
            __align__(16) __nv_bfloat16 w8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = kc * UK + grp * 8 + j;
                w8[j] = k < K ? W[(size_t)o * K + k] : __float2bfloat16(0.0f);
            }
            *reinterpret_cast<uint4*>(Bt + tile_off(o, grp * 8)) = *reinterpret_cast<const uint4*>(w8);
        }
        // generic-proxy writes of the tiles become visible to the tensor core
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_addr(A), b0 = smem_addr(Bt);
#pragma unroll
            for (int j = 0; j < UK / 16; ++j)
                umma_bf16(tmem, smem_desc(a0 + j * 2 * kLBO), smem_desc(b0 + j * 2 * kLBO), idesc,
                          (kc | j) != 0 ? 1u : 0u);
            umma_commit(&mbar[buf]);
        }
    }
    if (ok) ok = mbar_wait(&mbar[(nK - 1) & 1], (uint32_t)(((nK - 1) >> 1) & 1));
    if (!ok) {
        if (tid == 0) atomicExch(status, DEV_TIMEOUT);
        // let the MMAs already issued finish (bounded) before the accumulator is freed
        mbar_wait(&mbar[(nK - 1) & 1], (uint32_t)(((nK - 1) >> 1) & 1));
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        for (int o0 = 0; o0 < Cout; o0 += 16) {
            float v[16];
            tmem_ld16(trow + (uint32_t)o0, v);
            if (valid) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int o = o0 + i;
                    const size_t id = ((size_t)b * Cout + o) * npix + p;
                    const float z = v[i] + (bias ? bias[o] : 0.0f);
                    if (zout) zout[id] = z;
                    float y = relu ? fmaxf(z, 0.0f) : z;
                    if (gate && !(gate[id] > 0.0f)) y = 0.0f;
                    out[id] = y;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

}  // namespace

size_t conv3x3_umma_smem(int Cout) { return (size_t)2 * A_BYTES + (size_t)2 * Cout * UK * 2 + 2 * 8 + 16 + 1024; }

bool conv3x3_umma_ok(int Cin, int Cout) { return Cout % 16 == 0 && Cout >= 16 && Cout <= 256 && Cin >= 1; }

void conv3x3_umma(tt_ctx* c, int B, int Cin, int Cout, int nx, int ny, const float* X, const __nv_bfloat16* W,
                  const float* bias, int relu, const float* gate, float* zout, float* out) {
    TT_REQUIRE(conv3x3_umma_ok(Cin, Cout), "tensor-core convolution needs Cout %% 16 == 0, <= 256 (got %d)", Cout);
    const long long rows = (long long)B * nx * ny;
    const int grid = ceil_div(rows, UM);
    const size_t smem = conv3x3_umma_smem(Cout);
    CUDA_CHECK(cudaFuncSetAttribute(k_conv3x3_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope prof(c, PROF_CONV, 2.0 * 9 * Cin * Cout * (double)rows,
                   4.0 * (double)rows * (Cin + Cout * (zout ? 2 : 1)) + 2.0 * 9 * Cin * Cout);
    k_conv3x3_umma<<<grid, UM, smem, c->stream>>>(B, Cin, Cout, nx, ny, X, W, bias, relu, gate, zout, out,
                                                   c->dstatus);
    LAUNCH_CHECK(c);
}

}  // namespace tt
