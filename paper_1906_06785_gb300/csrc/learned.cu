// Learned mean-Oseen solve: a small convolutional network Phi on the lattice of
// velocity nodes approximates K^-1 r, K = tau^-1 M + A_0 + N(w_avg) the spatial
// factor of the inner preconditioner M of eq. (11_prec).  Inside M^-1 it replaces
// K^-1 on every column of the last core, so a train stays a train, and the
// flexible GMRES of Algorithm 4.2 (which stores the preconditioned vectors)
// absorbs its nonlinearity; the exact K^-1 stays the fallback.  The paper has no
// learned component: this is the extension, trained on the GPU by the kernels
// below on (r, K^-1 r) pairs from the exact banded solve.
//
// Network: 3x3 convolutions with zero padding, channels 5 -> C -> ... -> C -> 2,
// ReLU after every layer but the last.  Input channels: the residual's two
// components divided by its norm s, the two components of w_avg, the domain
// mask; output: the two components of the correction, read at the free nodes and
// multiplied by s.  Weights are held in FP32 (Adam's master copy) and used in
// BF16; every product accumulates in FP32, activations are FP32.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "solver.cuh"
#include "umma.cuh"

struct tt_net {
    tt_ctx* c = nullptr;          // context that owns the device buffers
    int nx = 0, ny = 0, npix = 0;
    int n_v = 0, n_nodes = 0;
    int C = 0, depth = 0;
    std::vector<int> cin, cout;   // per layer
    std::vector<size_t> woff, boff;
    size_t nparams = 0;
    tt::DBuf<int> pix_free;       // pixel -> free node index, or -1
    tt::DBuf<int> free_pix;       // free node index -> pixel
    tt::DBuf<int> node_pix;       // node -> pixel
    tt::DBuf<float> mask;         // npix
    tt::DBuf<float> theta;        // FP32 master parameters (per layer W then b)
    tt::DBuf<__nv_bfloat16> wb;   // BF16 weights, per layer [out][in][9]
    tt::DBuf<__nv_bfloat16> wflip;// BF16 weights of the transposed convolution [in][out][9]
    tt::DBuf<float> adam_m, adam_v;
    int adam_t = 0;
    // convolutions with at least 16 output channels run on the tcgen05 tensor cores
    // (BF16 activations as operands); 0: every convolution on the FP32 CUDA-core kernel
    int tensor_cores = 1;
};

namespace tt {
namespace {

constexpr int TILE = 16;   // output tile: TILE x TILE pixels
constexpr int OT = 16;     // output channels per block
constexpr int CC = 8;      // input channels staged per step

// ---------------------------------------------------------------- input features
// s[b] = ||column b|| of the n_u x ncol block Z (element (i, b) at Z[i * ldz + b]),
// with s = 1 for a zero column (the oracle's convention).
__global__ void k_col_scale(int n_u, int ncol, const double* __restrict__ Z, int ldz, float* __restrict__ s) {
    const int b = blockIdx.x;
    double a = 0.0;
    for (int i = threadIdx.x; i < n_u; i += blockDim.x) {
        const double v = Z[(size_t)i * ldz + b];
        a = fma(v, v, a);
    }
    __shared__ double red[32];
    a = warp_sum(a);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        a = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        a = warp_sum(a);
        if (threadIdx.x == 0) s[b] = a > 0.0 ? (float)sqrt(a) : 1.0f;
    }
}

// X[b][ch][p]: ch 0, 1 residual components / s_b at free nodes, 2, 3 w_avg, 4 mask.
__global__ void k_features(int ncol, int npix, int n_v, const int* __restrict__ pix_free,
                           const double* __restrict__ Z, int ldz, const float* __restrict__ s,
                           const float* __restrict__ wimg, const float* __restrict__ mask, float* __restrict__ X) {
    const long long tot = (long long)ncol * npix;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / npix), p = (int)(e % npix);
        const int f = pix_free[p];
        float* x = X + (size_t)b * 5 * npix;
        const float inv = 1.0f / s[b];
        x[p] = f >= 0 ? (float)Z[(size_t)f * ldz + b] * inv : 0.0f;
        x[npix + p] = f >= 0 ? (float)Z[(size_t)(n_v + f) * ldz + b] * inv : 0.0f;
        x[2 * npix + p] = wimg[p];
        x[3 * npix + p] = wimg[npix + p];
        x[4 * npix + p] = mask[p];
    }
}

// w_avg (2 n_nodes doubles) -> two lattice images (zero off the mesh)
__global__ void k_wimg(int n_nodes, int npix, const int* __restrict__ node_pix, const double* __restrict__ w,
                       float* __restrict__ img) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_nodes) return;
    img[node_pix[i]] = (float)w[i];
    img[npix + node_pix[i]] = (float)w[n_nodes + i];
}

// Y image (2 channels) -> out[(comp * n_v + i) * ldo + b] = s_b Y[b][comp][free_pix[i]]
__global__ void k_read_free(int ncol, int n_v, int npix, const int* __restrict__ free_pix,
                            const float* __restrict__ Y, const float* __restrict__ s, double* __restrict__ out,
                            int ldo) {
    const long long tot = 2LL * n_v * ncol;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e % ncol);
        const long long ci = e / ncol;
        const int comp = (int)(ci / n_v), i = (int)(ci % n_v);
        out[ci * ldo + b] = (double)s[b] * (double)Y[((size_t)b * 2 + comp) * npix + free_pix[i]];
    }
}

// ---------------------------------------------------------------- convolution
// out[b][o][p] = act(bias[o] + sum_{c, tap} W[o][c][tap] X[b][c][p + tap offset]) (zero
// padding), then, with a gate, out *= (gate[b][o][p] > 0).  W in BF16 [Cout][Cin][9],
// FP32 accumulation.  A block computes a TILE x TILE pixel tile of OT output channels
// of one image; Cin is staged CC channels at a time (halo tile + weights in shared
// memory).  With zout the pre-activation is stored too.
__global__ void __launch_bounds__(TILE * TILE)
k_conv3x3(int Cin, int Cout, int nx, int ny, const float* __restrict__ X, const __nv_bfloat16* __restrict__ W,
          const float* __restrict__ bias, int relu, const float* __restrict__ gate, float* __restrict__ zout,
          float* __restrict__ out) {
    __shared__ float xs[CC][TILE + 2][TILE + 2];
    __shared__ float ws[CC][9][OT];
    const int tiles_x = (nx + TILE - 1) / TILE;
    const int tx0 = (blockIdx.x % tiles_x) * TILE, ty0 = (blockIdx.x / tiles_x) * TILE;
    const int o0 = blockIdx.y * OT, b = blockIdx.z;
    const int tid = threadIdx.x, lx = tid % TILE, ly = tid / TILE;
    const int npix = nx * ny;
    const float* xb = X + (size_t)b * Cin * npix;
    float acc[OT];
#pragma unroll
    for (int k = 0; k < OT; ++k) acc[k] = 0.0f;
    for (int c0 = 0; c0 < Cin; c0 += CC) {
        for (int e = tid; e < CC * (TILE + 2) * (TILE + 2); e += TILE * TILE) {
            const int cc = e / ((TILE + 2) * (TILE + 2)), r = e % ((TILE + 2) * (TILE + 2));
            const int yy = ty0 - 1 + r / (TILE + 2), xx = tx0 - 1 + r % (TILE + 2);
            const int ch = c0 + cc;
            xs[cc][r / (TILE + 2)][r % (TILE + 2)] =
                (ch < Cin && yy >= 0 && yy < ny && xx >= 0 && xx < nx) ? xb[(size_t)ch * npix + yy * nx + xx] : 0.0f;
        }
        for (int e = tid; e < CC * 9 * OT; e += TILE * TILE) {
            const int k = e % OT, t = (e / OT) % 9, cc = e / (OT * 9);
            const int o = o0 + k, ch = c0 + cc;
            ws[cc][t][k] = (o < Cout && ch < Cin) ? __bfloat162float(W[((size_t)o * Cin + ch) * 9 + t]) : 0.0f;
        }
        __syncthreads();
        const int nc = min(CC, Cin - c0);
        for (int cc = 0; cc < nc; ++cc) {
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const float xv = xs[cc][ly + t / 3][lx + t % 3];
#pragma unroll
                for (int k = 0; k < OT; ++k) acc[k] = fmaf(ws[cc][t][k], xv, acc[k]);
            }
        }
        __syncthreads();
    }
    const int px = tx0 + lx, py = ty0 + ly;
    if (px >= nx || py >= ny) return;
    const int p = py * nx + px;
#pragma unroll
    for (int k = 0; k < OT; ++k) {
        const int o = o0 + k;
        if (o >= Cout) break;
        const size_t idx = ((size_t)b * Cout + o) * npix + p;
        float z = acc[k] + (bias ? bias[o] : 0.0f);
        if (zout) zout[idx] = z;
        float y = relu ? fmaxf(z, 0.0f) : z;
        if (gate && !(gate[idx] > 0.0f)) y = 0.0f;
        out[idx] = y;
    }
}

// gW[o][c][tap] += sum_b sum_p gY[b][o][p] X[b][c][p + tap offset]: a block owns an
// (OT x CC) channel pair block and a pixel tile, loops over the images, and adds its
// partial sums to gW.  Thread (o, c) of the block keeps 9 accumulators.
__global__ void __launch_bounds__(OT * CC)
k_conv3x3_wgrad(int B, int Cin, int Cout, int nx, int ny, const float* __restrict__ X,
                const float* __restrict__ gY, float* __restrict__ gW) {
    __shared__ float xs[CC][TILE + 2][TILE + 2];
    __shared__ float gs[OT][TILE * TILE];
    const int tiles_x = (nx + TILE - 1) / TILE;
    const int tx0 = (blockIdx.x % tiles_x) * TILE, ty0 = (blockIdx.x / tiles_x) * TILE;
    const int o0 = blockIdx.y * OT, c0 = blockIdx.z * CC;
    const int tid = threadIdx.x, ko = tid / CC, kc = tid % CC;
    const int npix = nx * ny;
    float acc[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[t] = 0.0f;
    for (int b = 0; b < B; ++b) {
        const float* xb = X + (size_t)b * Cin * npix;
        const float* gb = gY + (size_t)b * Cout * npix;
        for (int e = tid; e < CC * (TILE + 2) * (TILE + 2); e += OT * CC) {
            const int cc = e / ((TILE + 2) * (TILE + 2)), r = e % ((TILE + 2) * (TILE + 2));
            const int yy = ty0 - 1 + r / (TILE + 2), xx = tx0 - 1 + r % (TILE + 2);
            const int ch = c0 + cc;
            xs[cc][r / (TILE + 2)][r % (TILE + 2)] =
                (ch < Cin && yy >= 0 && yy < ny && xx >= 0 && xx < nx) ? xb[(size_t)ch * npix + yy * nx + xx] : 0.0f;
        }
        for (int e = tid; e < OT * TILE * TILE; e += OT * CC) {
            const int k = e / (TILE * TILE), r = e % (TILE * TILE);
            const int yy = ty0 + r / TILE, xx = tx0 + r % TILE, o = o0 + k;
            gs[k][r] = (o < Cout && yy < ny && xx < nx) ? gb[(size_t)o * npix + yy * nx + xx] : 0.0f;
        }
        __syncthreads();
        for (int ly = 0; ly < TILE; ++ly) {
#pragma unroll 4
            for (int lx = 0; lx < TILE; ++lx) {
                const float g = gs[ko][ly * TILE + lx];
#pragma unroll
                for (int t = 0; t < 9; ++t) acc[t] = fmaf(g, xs[kc][ly + t / 3][lx + t % 3], acc[t]);
            }
        }
        __syncthreads();
    }
    const int o = o0 + ko, ch = c0 + kc;
    if (o < Cout && ch < Cin)
        for (int t = 0; t < 9; ++t) atomicAdd(&gW[((size_t)o * Cin + ch) * 9 + t], acc[t]);
}

// gb[o] = sum_b sum_p gY[b][o][p]
__global__ void k_bias_grad(int B, int Cout, int npix, const float* __restrict__ gY, float* __restrict__ gb) {
    const int o = blockIdx.x;
    float a = 0.0f;
    for (long long e = threadIdx.x; e < (long long)B * npix; e += blockDim.x) {
        const int b = (int)(e / npix), p = (int)(e % npix);
        a += gY[((size_t)b * Cout + o) * npix + p];
    }
    a = warp_sum(a);
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        a = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        a = warp_sum(a);
        if (threadIdx.x == 0) gb[o] = a;
    }
}

// Training loss of a batch of (r, t) pairs: per column b, e = s_b Y[b][:, free] - t_b,
// loss += ||e||^2 / ||t_b||^2 / B and gY[b][comp][free_pix[i]] = 2 e_i s_b / (||t_b||^2 B)
// (gY zero elsewhere, set by the caller).  One block per column.
__global__ void k_loss(int B, int n_v, int npix, const int* __restrict__ free_pix, const float* __restrict__ Y,
                       const float* __restrict__ s, const double* __restrict__ T, int ldt,
                       float* __restrict__ gY, double* __restrict__ loss) {
    const int b = blockIdx.x;
    __shared__ double red[32];
    __shared__ double den_s;
    double d = 0.0;
    for (int i = threadIdx.x; i < 2 * n_v; i += blockDim.x) {
        const double t = T[(size_t)i * ldt + b];
        d = fma(t, t, d);
    }
    d = warp_sum(d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x < 32) {
        d = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        d = warp_sum(d);
        if (threadIdx.x == 0) den_s = d > 0.0 ? d : 1.0;
    }
    __syncthreads();
    const double den = den_s;
    const double sb = s[b];
    double l = 0.0;
    for (int i = threadIdx.x; i < 2 * n_v; i += blockDim.x) {
        const int comp = i / n_v, f = i % n_v;
        const size_t yi = ((size_t)b * 2 + comp) * npix + free_pix[f];
        const double e = sb * (double)Y[yi] - T[(size_t)i * ldt + b];
        l = fma(e, e, l);
        gY[yi] = (float)(2.0 * e * sb / (den * B));
    }
    __syncthreads();
    l = warp_sum(l);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x < 32) {
        l = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        l = warp_sum(l);
        if (threadIdx.x == 0) atomicAdd(loss, l / den / B);
    }
}

// BF16 copies of the weights of every layer: wb[o][c][t] and the transposed, flipped
// filter of the backward convolution wflip[c][o][8 - t].
__global__ void k_weights_bf16(int n, const float* __restrict__ W, int Cin, int Cout, __nv_bfloat16* __restrict__ wb,
                               __nv_bfloat16* __restrict__ wflip) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int t = e % 9, oc = e / 9, c = oc % Cin, o = oc / Cin;
    const __nv_bfloat16 v = __float2bfloat16(W[e]);
    wb[e] = v;
    wflip[((size_t)c * Cout + o) * 9 + (8 - t)] = v;
}

// Adam (Kingma and Ba, 2015) on the flat FP32 parameters: bias-corrected moments,
// theta -= lr m_hat / (sqrt(v_hat) + eps).
__global__ void k_adam(int n, float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    theta[i] -= lr * mh / (sqrtf(vh) + eps);
}

// y = x - omega D^-1 (K x) for the two components of ncol columns (weighted Jacobi),
// Kx given; D the diagonal of K (ff slots diag_slot).
__global__ void k_jacobi_smooth(int n_v, int ncol, const double* __restrict__ kv, const int* __restrict__ diag_slot,
                                const double* __restrict__ KX, int ldk, double omega, double* __restrict__ X,
                                int ldx) {
    const long long tot = 2LL * n_v * ncol;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e % ncol);
        const long long ci = e / ncol;
        const int i = (int)(ci % n_v);
        X[ci * ldx + b] -= omega * KX[ci * ldk + b] / kv[diag_slot[i]];
    }
}
}  // namespace

// ---------------------------------------------------------------- host side
namespace {
void refresh_weights(tt_ctx* c, tt_net* net) {
    for (int l = 0; l < net->depth; ++l) {
        const int n = net->cout[l] * net->cin[l] * 9;
        k_weights_bf16<<<ceil_div(n, 256), 256, 0, c->stream>>>(n, net->theta.p + net->woff[l], net->cin[l],
                                                                  net->cout[l], net->wb.p + net->woff[l],
                                                                  net->wflip.p + net->woff[l]);
        LAUNCH_CHECK(c);
    }
}

void conv_launch(tt_ctx* c, const tt_net* net, int B, int Cin, int Cout, const float* X, const __nv_bfloat16* W,
                 const float* bias, int relu, const float* gate, float* zout, float* out) {
    if (net->tensor_cores && conv3x3_umma_ok(Cin, Cout)) {
        conv3x3_umma(c, B, Cin, Cout, net->nx, net->ny, X, W, bias, relu, gate, zout, out);
        return;
    }
    const int tiles = ceil_div(net->nx, TILE) * ceil_div(net->ny, TILE);
    ProfScope prof(c, PROF_CONV, 2.0 * 9 * Cin * Cout * (double)net->npix * B,
                   4.0 * ((double)B * (Cin + Cout * (zout ? 2 : 1)) * net->npix) + 2.0 * 9 * Cin * Cout);
    k_conv3x3<<<dim3(tiles, ceil_div(Cout, OT), B), TILE * TILE, 0, c->stream>>>(Cin, Cout, net->nx, net->ny, X, W,
                                                                                 bias, relu, gate, zout, out);
    LAUNCH_CHECK(c);
}

// Work buffers of one pass over B columns: layer inputs H[l] (H[0] = features) and
// pre-activations Z[l], output image, scales.
struct NetPass {
    std::vector<DBuf<float>> H, Z;
    DBuf<float> s, wimg;
    NetPass(tt_ctx* c, const tt_net* net, int B, bool keep) {
        H.resize(net->depth + 1);
        Z.resize(net->depth);
        for (int l = 0; l <= net->depth; ++l) {
            const int ch = l == 0 ? net->cin[0] : net->cout[l - 1];
            if (keep || l == 0 || l == net->depth || l <= 2) H[l].alloc(c, (size_t)B * ch * net->npix);
        }
        if (keep)
            for (int l = 0; l < net->depth; ++l) Z[l].alloc(c, (size_t)B * net->cout[l] * net->npix);
        s.alloc(c, B);
        wimg.alloc(c, 2 * (size_t)net->npix);
    }
};

// Forward pass of B columns of Z (n_u x B block at stride ldz): features, layers.
// keep: store every layer input and pre-activation (training); else ping-pong.
const float* net_forward(tt_ctx* c, const tt_net* net, NetPass& w, int B, const double* Z, int ldz,
                         const double* wavg, bool keep) {
    k_col_scale<<<B, 256, 0, c->stream>>>(2 * net->n_v, B, Z, ldz, w.s.p);
    LAUNCH_CHECK(c);
    CUDA_CHECK(cudaMemsetAsync(w.wimg.p, 0, 2 * (size_t)net->npix * sizeof(float), c->stream));
    k_wimg<<<ceil_div(net->n_nodes, 256), 256, 0, c->stream>>>(net->n_nodes, net->npix, net->node_pix.p, wavg,
                                                                w.wimg.p);
    LAUNCH_CHECK(c);
    const long long tot = (long long)B * net->npix;
    k_features<<<(int)std::min<long long>(4096, (tot + 255) / 256), 256, 0, c->stream>>>(
        B, net->npix, net->n_v, net->pix_free.p, Z, ldz, w.s.p, w.wimg.p, net->mask.p, w.H[0].p);
    LAUNCH_CHECK(c);
    const float* in = w.H[0].p;
    for (int l = 0; l < net->depth; ++l) {
        const bool last = l == net->depth - 1;
        float* out = keep || last ? w.H[l + 1].p : w.H[1 + (l % 2)].p;
        conv_launch(c, net, B, net->cin[l], net->cout[l], in, net->wb.p + net->woff[l], net->theta.p + net->boff[l],
                    last ? 0 : 1, nullptr, keep ? w.Z[l].p : nullptr, out);
        in = out;
    }
    return in;
}
}  // namespace

namespace {
__global__ void k_cumsum_time(int n_t, int r, const double* __restrict__ in, double* __restrict__ out) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= r) return;
    double s = 0.0;
    for (int t = 0; t < n_t; ++t) {
        s += in[(size_t)a * n_t + t];
        out[(size_t)a * n_t + t] = s;
    }
}

// Phi applied to the n_u x ncol block Z (row stride ldz) into out (row stride ldo),
// in chunks of at most kChunk columns.
constexpr int kChunk = 128;
void net_apply_block(tt_ctx* c, const tt_net* net, const double* wavg, const double* Z, int ldz, int ncol,
                     double* out, int ldo) {
    const int B = std::min(ncol, kChunk);
    NetPass w(c, net, B, false);
    for (int b0 = 0; b0 < ncol; b0 += B) {
        const int nb = std::min(B, ncol - b0);
        const float* Y = net_forward(c, net, w, nb, Z + b0, ldz, wavg, false);
        k_read_free<<<(int)std::min<long long>(4096, (2LL * net->n_v * nb + 255) / 256), 256, 0, c->stream>>>(
            nb, net->n_v, net->npix, net->free_pix.p, Y, w.s.p, out + b0, ldo);
        LAUNCH_CHECK(c);
    }
}

// Loss and gradients (into grad, nparams floats, zeroed here) of one batch of B pairs
// whose residuals and targets are n_u x B blocks (row strides ldr, ldt).
double net_loss_grad(tt_ctx* c, tt_net* net, NetPass& w, int B, const double* wavg, const double* R, int ldr,
                     const double* T, int ldt, float* grad, double* dloss) {
    const int L = net->depth;
    const float* Y = net_forward(c, net, w, B, R, ldr, wavg, true);
    (void)Y;
    const size_t img = (size_t)B * net->C * net->npix;
    DBuf<float> g0(c, std::max(img, (size_t)B * 2 * net->npix)), g1(c, img);
    CUDA_CHECK(cudaMemsetAsync(g0.p, 0, (size_t)B * 2 * net->npix * sizeof(float), c->stream));
    CUDA_CHECK(cudaMemsetAsync(grad, 0, net->nparams * sizeof(float), c->stream));
    CUDA_CHECK(cudaMemsetAsync(dloss, 0, sizeof(double), c->stream));
    k_loss<<<B, 256, 0, c->stream>>>(B, net->n_v, net->npix, net->free_pix.p, w.H[L].p, w.s.p, T, ldt, g0.p, dloss);
    LAUNCH_CHECK(c);
    float* g = g0.p;
    float* gn = g1.p;
    const int tiles = ceil_div(net->nx, TILE) * ceil_div(net->ny, TILE);
    for (int l = L - 1; l >= 0; --l) {
        const int ci = net->cin[l], co = net->cout[l];
        {
            ProfScope prof(c, PROF_CONV, 2.0 * 9 * ci * co * (double)net->npix * B,
                           4.0 * (double)B * (ci + co) * net->npix);
            k_conv3x3_wgrad<<<dim3(tiles, ceil_div(co, OT), ceil_div(ci, CC)), OT * CC, 0, c->stream>>>(
                B, ci, co, net->nx, net->ny, w.H[l].p, g, grad + net->woff[l]);
            LAUNCH_CHECK(c);
        }
        k_bias_grad<<<co, 256, 0, c->stream>>>(B, co, net->npix, g, grad + net->boff[l]);
        LAUNCH_CHECK(c);
        if (l > 0) {
            // gradient of the layer input, gated by the ReLU of the layer below
            conv_launch(c, net, B, co, ci, g, net->wflip.p + net->woff[l], nullptr, 0, w.Z[l - 1].p, nullptr, gn);
            std::swap(g, gn);
        }
    }
    double h = 0.0;
    read_back(c, (const double*)dloss, &h, 1);
    return h;
}
}  // namespace

TTPtr learned_minv(tt_ctx* c, const tt_net* net, tt_op* op, const tt_t* z) {
    tt_problem* P = op->P;
    TT_REQUIRE(net->n_v == P->n_v && net->n_nodes == P->n_nodes, "network built for another mesh");
    TT_REQUIRE(z->n_x == 2 * P->n_v, "learned M^-1 applies to velocity trains");
    TTPtr out = wrap(tt_alloc(c, z->n_t, z->n_xi, z->n_x, z->r1, z->r2));
    k_cumsum_time<<<ceil_div(z->r1, 64), 64, 0, c->stream>>>(z->n_t, z->r1, z->z1, out->z1);
    LAUNCH_CHECK(c);
    CUDA_CHECK(cudaMemcpyAsync(out->z2, z->z2, (size_t)z->r1 * z->n_xi * z->r2 * sizeof(double),
                               cudaMemcpyDeviceToDevice, c->stream));
    DBuf<double> wavg(c, 2 * (size_t)P->n_nodes);
    op_wavg(c, op, wavg.p);
    net_apply_block(c, net, wavg.p, z->z3, z->r2, z->r2, out->z3, z->r2);
    return out;
}

}  // namespace tt

using namespace tt;

#define NET_API_BEGIN(ctx) \
    tt_ctx* _ctx = (ctx);  \
    try {
#define NET_API_END                     \
    return TT_OK;                       \
    }                                   \
    catch (const tt::Error& e) {        \
        if (_ctx) _ctx->err = e.what(); \
        return e.code;                  \
    }                                   \
    catch (const std::exception& e) {   \
        if (_ctx) _ctx->err = e.what(); \
        return TT_ECUDA;                \
    }

namespace {
// host (or device) double block -> device, as an n_u x count row-major block
void upload_block(tt_ctx* c, DBuf<double>& dst, const double* src, size_t n, int on_device) {
    dst.alloc(c, n);
    CUDA_CHECK(cudaMemcpyAsync(dst.p, src, n * sizeof(double),
                               on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
}
void check_net_op(const tt_net* net, const tt_op* op) {
    TT_REQUIRE(op->which == TT_OP_FULL, "the network needs a FULL operator (its convection field)");
    TT_REQUIRE(net->n_v == op->P->n_v && net->n_nodes == op->P->n_nodes, "network built for another mesh");
}
}  // namespace

extern "C" {

int tt_net_create(tt_ctx* ctx, const tt_problem* P, int channels, int depth, const float* params, tt_net** out) {
    NET_API_BEGIN(ctx)
    TT_REQUIRE(ctx && P && params && out, "null argument");
    TT_REQUIRE(channels >= 1 && channels <= 512 && depth >= 2 && depth <= 16, "bad network size C=%d depth=%d",
               channels, depth);
    *out = nullptr;
    std::unique_ptr<tt_net> net(new tt_net);
    net->c = ctx;
    net->C = channels;
    net->depth = depth;
    net->n_v = P->n_v;
    net->n_nodes = P->n_nodes;
    // lattice of the velocity nodes: spacing h/2 from the lower-left corner
    const int n = P->n_nodes;
    double x0 = 1e300, y0 = 1e300;
    for (int i = 0; i < n; ++i) {
        x0 = std::min(x0, P->hxy[2 * i]);
        y0 = std::min(y0, P->hxy[2 * i + 1]);
    }
    const double hv = P->h / 2.0;
    std::vector<int> ix(n), iy(n);
    int nx = 0, ny = 0;
    for (int i = 0; i < n; ++i) {
        ix[i] = (int)std::lround((P->hxy[2 * i] - x0) / hv);
        iy[i] = (int)std::lround((P->hxy[2 * i + 1] - y0) / hv);
        nx = std::max(nx, ix[i] + 1);
        ny = std::max(ny, iy[i] + 1);
    }
    net->nx = nx;
    net->ny = ny;
    net->npix = nx * ny;
    std::vector<int> pix_free(net->npix, -1), free_pix(P->n_v), node_pix(n);
    std::vector<float> mask(net->npix, 0.0f);
    for (int i = 0; i < n; ++i) {
        const int p = iy[i] * nx + ix[i];
        node_pix[i] = p;
        mask[p] = 1.0f;
        if (P->fidx[i] >= 0) {
            free_pix[P->fidx[i]] = p;
            pix_free[p] = P->fidx[i];
        }
    }
    net->pix_free.alloc(ctx, net->npix);
    net->free_pix.alloc(ctx, P->n_v);
    net->node_pix.alloc(ctx, n);
    net->mask.alloc(ctx, net->npix);
    CUDA_CHECK(cudaMemcpyAsync(net->pix_free.p, pix_free.data(), pix_free.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CUDA_CHECK(cudaMemcpyAsync(net->free_pix.p, free_pix.data(), free_pix.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CUDA_CHECK(cudaMemcpyAsync(net->node_pix.p, node_pix.data(), node_pix.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CUDA_CHECK(cudaMemcpyAsync(net->mask.p, mask.data(), mask.size() * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    size_t off = 0;
    for (int l = 0; l < depth; ++l) {
        net->cin.push_back(l == 0 ? 5 : channels);
        net->cout.push_back(l == depth - 1 ? 2 : channels);
        net->woff.push_back(off);
        off += (size_t)net->cout[l] * net->cin[l] * 9;
        net->boff.push_back(off);
        off += net->cout[l];
    }
    net->nparams = off;
    net->theta.alloc(ctx, off);
    net->wb.alloc(ctx, off);
    net->wflip.alloc(ctx, off);
    net->adam_m.alloc(ctx, off);
    net->adam_v.alloc(ctx, off);
    CUDA_CHECK(cudaMemcpyAsync(net->theta.p, params, off * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    CUDA_CHECK(cudaMemsetAsync(net->adam_m.p, 0, off * sizeof(float), ctx->stream));
    CUDA_CHECK(cudaMemsetAsync(net->adam_v.p, 0, off * sizeof(float), ctx->stream));
    refresh_weights(ctx, net.get());
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    *out = net.release();
    NET_API_END
}

int tt_net_destroy(tt_net* net) {
    if (!net) return TT_EINVAL;
    delete net;
    return TT_OK;
}

int tt_net_set_tensor_cores(tt_net* net, int on) {
    if (!net) return TT_EINVAL;
    net->tensor_cores = on ? 1 : 0;
    return TT_OK;
}

int tt_net_info(const tt_net* net, int* nparams, int* nx, int* ny) {
    if (!net) return TT_EINVAL;
    if (nparams) *nparams = (int)net->nparams;
    if (nx) *nx = net->nx;
    if (ny) *ny = net->ny;
    return TT_OK;
}

int tt_net_get_params(tt_ctx* ctx, const tt_net* net, float* params) {
    NET_API_BEGIN(ctx)
    TT_REQUIRE(ctx && net && params, "null argument");
    CUDA_CHECK(cudaMemcpyAsync(params, net->theta.p, net->nparams * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    NET_API_END
}

int tt_net_apply(tt_ctx* ctx, const tt_net* net, const tt_op* op, const double* R, int count, int on_device,
                 double* out) {
    NET_API_BEGIN(ctx)
    TT_REQUIRE(ctx && net && op && R && out && count > 0, "bad argument");
    check_net_op(net, op);
    const size_t n = (size_t)2 * net->n_v * count;
    DBuf<double> dR, dO(ctx, n);
    upload_block(ctx, dR, R, n, on_device);
    DBuf<double> wavg(ctx, 2 * (size_t)net->n_nodes);
    op_wavg(ctx, op, wavg.p);
    net_apply_block(ctx, net, wavg.p, dR.p, count, count, dO.p, count);
    CUDA_CHECK(cudaMemcpyAsync(out, dO.p, n * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                               ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    NET_API_END
}

int tt_net_loss_grad(tt_ctx* ctx, tt_net* net, const tt_op* op, const double* R, const double* T, int count,
                     int on_device, double* loss, float* grads) {
    NET_API_BEGIN(ctx)
    TT_REQUIRE(ctx && net && op && R && T && count > 0, "bad argument");
    check_net_op(net, op);
    const size_t n = (size_t)2 * net->n_v * count;
    DBuf<double> dR, dT;
    upload_block(ctx, dR, R, n, on_device);
    upload_block(ctx, dT, T, n, on_device);
    DBuf<double> wavg(ctx, 2 * (size_t)net->n_nodes), dl(ctx, 1);
    op_wavg(ctx, op, wavg.p);
    DBuf<float> g(ctx, net->nparams);
    NetPass w(ctx, net, count, true);
    const double l = net_loss_grad(ctx, net, w, count, wavg.p, dR.p, count, dT.p, count, g.p, dl.p);
    if (loss) *loss = l;
    if (grads) {
        CUDA_CHECK(cudaMemcpyAsync(grads, g.p, net->nparams * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
        CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    }
    NET_API_END
}

int tt_net_train(tt_ctx* ctx, tt_net* net, tt_op* op, const double* R, int count, int on_device,
                 const tt_train_opts* o, double* epoch_loss) {
    NET_API_BEGIN(ctx)
    TT_REQUIRE(ctx && net && op && R && o && count > 0, "bad argument");
    check_net_op(net, op);
    TT_REQUIRE(o->batch >= 1 && o->epochs >= 0 && o->smooth_max >= 0 && o->lr > 0.0f, "bad training options");
    tt_problem* P = op->P;
    const int nv = net->n_v;
    const size_t n = (size_t)2 * nv * count;
    // residuals, smoothed in contiguous groups by 0 .. smooth_max weighted-Jacobi sweeps of K
    DBuf<double> dR, dT(ctx, n);
    upload_block(ctx, dR, R, n, on_device);
    DBuf<double> wavg(ctx, 2 * (size_t)P->n_nodes), dl(ctx, 1);
    const bool has_w = op_wavg(ctx, op, wavg.p);
    if (o->smooth_max > 0) {
        DBuf<double> kv(ctx, P->ff.nnz), KX(ctx, n);
        assemble_K_vals(ctx, P, has_w ? wavg.p : nullptr, kv.p);
        for (int j = 1; j <= o->smooth_max; ++j) {
            const int start = (int)(((long long)j * count + o->smooth_max) / (o->smooth_max + 1));
            if (start >= count) break;
            VelSpmm s{};
            s.rowptr = P->ff.rowptr.p; s.col = P->ff.col.p; s.n_rows = nv; s.n_in = nv; s.nnz = P->ff.nnz;
            s.ncomp = 2;
            s.nmat = 1; s.vals[0] = kv.p; s.coef[0] = 1.0; s.coff[0] = 0;
            PrecScope fp64(ctx, 0);
            spmm_vel(ctx, s, dR.p + start, count, KX.p + start, count, count - start);
            k_jacobi_smooth<<<(int)std::min<long long>(4096, (2LL * nv * (count - start) + 255) / 256), 256, 0,
                              ctx->stream>>>(nv, count - start, kv.p, P->diag_slot.p, KX.p + start, count,
                                             (double)o->omega, dR.p + start, count);
            LAUNCH_CHECK(ctx);
        }
    }
    // targets t = K^-1 r by the exact banded solve (FP64)
    op_ensure_K(ctx, op);
    CUDA_CHECK(cudaMemcpyAsync(dT.p, dR.p, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    {
        PrecScope fp64(ctx, 0);
        band_solve(ctx, op->Kband.p, nv, P->bwK, dT.p, count, count, 2);
    }
    const int B = std::min(o->batch, count);
    DBuf<float> g(ctx, net->nparams);
    NetPass w(ctx, net, B, true);
    for (int ep = 0; ep < o->epochs; ++ep) {
        double tot = 0.0;
        int nb = 0;
        for (int b0 = 0; b0 + B <= count; b0 += B) {
            tot += net_loss_grad(ctx, net, w, B, wavg.p, dR.p + b0, count, dT.p + b0, count, g.p, dl.p);
            ++nb;
            net->adam_t += 1;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.0f - std::pow(b1, (float)net->adam_t), c2 = 1.0f - std::pow(b2, (float)net->adam_t);
            k_adam<<<ceil_div((long long)net->nparams, 256), 256, 0, ctx->stream>>>(
                (int)net->nparams, net->theta.p, g.p, net->adam_m.p, net->adam_v.p, o->lr, b1, b2, 1e-8f, c1, c2);
            LAUNCH_CHECK(ctx);
            refresh_weights(ctx, net);
        }
        if (epoch_loss) epoch_loss[ep] = nb ? tot / nb : 0.0;
    }
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    NET_API_END
}

}  // extern "C"
