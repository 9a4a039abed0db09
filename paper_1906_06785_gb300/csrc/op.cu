// Operators of the all-at-once system as sums of Kronecker products applied to
// trains (eq. Xz): every term acts on the first core in time (identity, shift
// C_{n_t}, diagonal, cumulative sum), on the middle core with an n_xi x n_xi
// gPC matrix, and on the last core with a sparse spatial operator.  Terms that
// share a time operator and input share a core-1 block; terms that share a
// spatial operator and input share a core-3 block; the middle core is block
// sparse.  Spatial products of one input over the shared Q2 pattern run as
// one multi-matrix SpMM launch.
#include <algorithm>
#include <cmath>
#include <map>

#include "op.cuh"

namespace tt {

namespace {
struct Dev1 {
    const double* in;
    const double* vec;
    int kind, r, off;
};
// out1[(off + a) * n_t + t]
__global__ void k_core1(const Dev1* __restrict__ B, int n_t, double* __restrict__ out) {
    const Dev1 q = B[blockIdx.y];
    if (q.kind == T_CUMSUM) {
        for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < q.r; a += gridDim.x * blockDim.x) {
            double s = 0.0;
            for (int t = 0; t < n_t; ++t) {
                s += q.in[(size_t)a * n_t + t];
                out[(size_t)(q.off + a) * n_t + t] = s;
            }
        }
        return;
    }
    const int tot = n_t * q.r;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
        const int t = e % n_t;
        double v;
        if (q.kind == T_COPY) v = q.in[e];
        else if (q.kind == T_SHIFT) v = t > 0 ? q.in[e - 1] : 0.0;
        else v = q.vec[t] * q.in[e];
        out[(size_t)q.off * n_t + e] = v;
    }
}

struct Dev2 {
    const double* in;
    const double* S;
    const double* dcoef;
    double coef;
    int r1, r2, off1, off3;
};
// out2[((off1 + a) * n_xi + s) * R2 + off3 + b] += cf * sum_r S[s][r] in[(a n_xi + r) r2 + b]
__global__ void k_core2(const Dev2* __restrict__ T, int n_xi, int R2, double* __restrict__ out) {
    const Dev2 q = T[blockIdx.y];
    const double cf = q.coef * (q.dcoef ? *q.dcoef : 1.0);
    const long long tot = (long long)q.r1 * n_xi * q.r2;
    for (long long e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e % q.r2);
        const long long as = e / q.r2;
        const int s = (int)(as % n_xi), a = (int)(as / n_xi);
        double v;
        if (q.S) {
            v = 0.0;
            const double* Srow = q.S + (size_t)s * n_xi;
            const double* col = q.in + (size_t)a * n_xi * q.r2 + b;
            for (int r = 0; r < n_xi; ++r) v = fma(Srow[r], col[(size_t)r * q.r2], v);
        } else {
            v = q.in[e];
        }
        out[((size_t)(q.off1 + a) * n_xi + s) * R2 + q.off3 + b] += cf * v;
    }
}

// copy a core-3 block with optional per-row velocity scaling 1/d (both components)
__global__ void k_core3_copy(int rows, int r, const double* __restrict__ in, double* __restrict__ out, int R2, int off,
                             double coef, const double* __restrict__ dinv, int n_v) {
    const long long tot = (long long)rows * r;
    for (long long e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e % r);
        const long long i = e / r;
        double v = coef * in[e];
        if (dinv) v /= dinv[i % n_v];
        out[i * R2 + off + b] = v;
    }
}

// embed rows: out[(c * n_nodes + map[i]) * R2 + off + b] = in[(c * n_in + i) * r + b]
__global__ void k_embed(int n_in, int n_nodes, int r, const int* __restrict__ map, const double* __restrict__ in,
                        double* __restrict__ out, int R2, int off) {
    const long long tot = 2LL * n_in * r;
    for (long long e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e % r);
        const long long ci = e / r;
        const int c = (int)(ci / n_in), i = (int)(ci % n_in);
        out[((size_t)c * n_nodes + map[i]) * R2 + off + b] = in[e];
    }
}
}  // namespace

static int out_rows(tt_problem* P, SKind k, const tt_t* in) {
    switch (k) {
        case S_COPY: case S_MSTARINV: case S_SOLVE_K: case S_SOLVE_LP: case S_MPSTARINV: return in->n_x;
        case S_PRES: return P->n_p;
        case S_VEL: case S_VELD: case S_GRAD: return 2 * P->n_v;
        case S_DIV: case S_DIVD: return P->n_p;
        case S_EMBED_F: case S_EMBED_D: return 2 * P->n_nodes;
    }
    return -1;
}

static void check_in_rows(tt_problem* P, SKind k, const tt_t* in) {
    int need = -1;
    switch (k) {
        case S_VEL: case S_DIV: case S_MSTARINV: case S_SOLVE_K: case S_EMBED_F: need = 2 * P->n_v; break;
        case S_VELD: case S_DIVD: case S_EMBED_D: need = 2 * P->n_D; break;
        case S_GRAD: case S_SOLVE_LP: case S_PRES: case S_MPSTARINV: need = P->n_p; break;
        default: break;
    }
    TT_REQUIRE(need < 0 || in->n_x == need, "spatial operator %d expects %d rows, train has %d", (int)k, need, in->n_x);
}

TTPtr kron_sum(tt_ctx* c, tt_problem* P, const std::vector<C1>& b1, const std::vector<C3>& b3,
               const std::vector<C2>& b2) {
    TT_REQUIRE(!b1.empty() && !b3.empty() && !b2.empty(), "empty Kronecker sum");
    const int n_t = b1[0].in->n_t, n_xi = b1[0].in->n_xi;
    const int n_x = out_rows(P, b3[0].kind, b3[0].in);
    std::vector<int> off1(b1.size()), off3(b3.size());
    int R1 = 0, R2 = 0;
    for (size_t i = 0; i < b1.size(); ++i) {
        TT_REQUIRE(b1[i].in->n_t == n_t && b1[i].in->n_xi == n_xi, "core-1 block shape mismatch");
        off1[i] = R1;
        R1 += b1[i].in->r1;
    }
    for (size_t i = 0; i < b3.size(); ++i) {
        check_in_rows(P, b3[i].kind, b3[i].in);
        TT_REQUIRE(out_rows(P, b3[i].kind, b3[i].in) == n_x, "core-3 blocks of different sizes");
        off3[i] = R2;
        R2 += b3[i].in->r2;
    }
    for (auto& q : b2) {
        TT_REQUIRE(q.b1 >= 0 && q.b1 < (int)b1.size() && q.b3 >= 0 && q.b3 < (int)b3.size(), "bad core-2 term");
        TT_REQUIRE(b1[q.b1].in == b3[q.b3].in, "core-2 term joins blocks of different inputs");
    }
    TTPtr out = wrap(tt_alloc(c, n_t, n_xi, n_x, R1, R2));

    // ---- core 1
    {
        std::vector<Dev1> h(b1.size());
        int maxr = 1;
        for (size_t i = 0; i < b1.size(); ++i) {
            h[i] = Dev1{b1[i].in->z1, b1[i].vec, (int)b1[i].kind, b1[i].in->r1, off1[i]};
            maxr = std::max(maxr, b1[i].in->r1);
        }
        DBuf<Dev1> d(c, h.size());
        CUDA_CHECK(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(Dev1), cudaMemcpyHostToDevice, c->stream));
        k_core1<<<dim3(ceil_div((long long)n_t * maxr, 256), (unsigned)h.size()), 256, 0, c->stream>>>(d.p, n_t, out->z1);
        LAUNCH_CHECK(c);
    }
    // ---- core 2 (block sparse; terms on the same block are applied in separate launches)
    {
        fill_zero(c, out->z2, (size_t)R1 * n_xi * R2);
        std::vector<std::vector<Dev2>> waves;
        std::vector<std::map<std::pair<int, int>, int>> used;
        for (auto& q : b2) {
            const tt_t* in = b1[q.b1].in;
            Dev2 d{in->z2, q.S, q.dcoef, q.coef, in->r1, in->r2, off1[q.b1], off3[q.b3]};
            size_t w = 0;
            while (w < waves.size() && used[w].count({q.b1, q.b3})) ++w;
            if (w == waves.size()) { waves.emplace_back(); used.emplace_back(); }
            waves[w].push_back(d);
            used[w][{q.b1, q.b3}] = 1;
        }
        for (auto& wv : waves) {
            DBuf<Dev2> d(c, wv.size());
            CUDA_CHECK(cudaMemcpyAsync(d.p, wv.data(), wv.size() * sizeof(Dev2), cudaMemcpyHostToDevice, c->stream));
            long long maxe = 1;
            for (auto& q : wv) maxe = std::max(maxe, (long long)q.r1 * n_xi * q.r2);
            k_core2<<<dim3(std::min(1024, ceil_div(maxe, 256)), (unsigned)wv.size()), 256, 0, c->stream>>>(
                d.p, n_xi, R2, out->z2);
            LAUNCH_CHECK(c);
        }
    }
    // ---- core 3: group S_VEL / S_VELD blocks of one input into multi-matrix launches
    {
        std::vector<bool> done(b3.size(), false);
        for (size_t i = 0; i < b3.size(); ++i) {
            if (done[i]) continue;
            const C3& q = b3[i];
            const tt_t* in = q.in;
            if (q.kind == S_VEL || q.kind == S_VELD || q.kind == S_PRES) {
                const Csr& pat = q.kind == S_VEL ? P->ff : q.kind == S_VELD ? P->fD : P->pp;
                VelSpmm s{};
                s.rowptr = pat.rowptr.p; s.col = pat.col.p; s.nnz = pat.nnz;
                s.n_rows = q.kind == S_PRES ? P->n_p : P->n_v;
                s.n_in = q.kind == S_VEL ? P->n_v : q.kind == S_VELD ? P->n_D : P->n_p;
                s.ncomp = q.kind == S_PRES ? 1 : 2;
                s.nmat = 0;
                for (size_t j = i; j < b3.size(); ++j) {
                    if (done[j] || b3[j].in != in || b3[j].kind != q.kind) continue;
                    s.vals[s.nmat] = b3[j].vals; s.coef[s.nmat] = b3[j].coef; s.coff[s.nmat] = off3[j];
                    ++s.nmat;
                    done[j] = true;
                    if (s.nmat == 8) {
                        spmm_vel(c, s, in->z3, in->r2, out->z3, R2, in->r2);
                        s.nmat = 0;
                    }
                }
                if (s.nmat) spmm_vel(c, s, in->z3, in->r2, out->z3, R2, in->r2);
                continue;
            }
            done[i] = true;
            const long long tot = (long long)in->n_x * in->r2;
            switch (q.kind) {
                case S_COPY:
                case S_MSTARINV:
                case S_MPSTARINV:
                    k_core3_copy<<<std::min(4096, ceil_div(tot, 256)), 256, 0, c->stream>>>(
                        in->n_x, in->r2, in->z3, out->z3, R2, off3[i], q.coef,
                        q.kind == S_MSTARINV ? P->Mstar.p : q.kind == S_MPSTARINV ? P->Mpstar.p : nullptr,
                        q.kind == S_MPSTARINV ? P->n_p : P->n_v);
                    LAUNCH_CHECK(c);
                    break;
                case S_DIV:
                    spmm_div(c, P->BF, P->Bx_F.p, P->By_F.p, P->n_v, q.coef, in->z3, in->r2, out->z3, R2, off3[i], in->r2);
                    break;
                case S_DIVD:
                    spmm_div(c, P->BD, P->Bx_D.p, P->By_D.p, P->n_D, q.coef, in->z3, in->r2, out->z3, R2, off3[i], in->r2);
                    break;
                case S_GRAD:
                    spmm_grad(c, P->BT, P->BTx.p, P->BTy.p, q.coef, in->z3, in->r2, out->z3, R2, off3[i], in->r2);
                    break;
                case S_SOLVE_K:
                case S_SOLVE_LP: {
                    k_core3_copy<<<std::min(4096, ceil_div(tot, 256)), 256, 0, c->stream>>>(
                        in->n_x, in->r2, in->z3, out->z3, R2, off3[i], q.coef, nullptr, 1);
                    LAUNCH_CHECK(c);
                    if (q.kind == S_SOLVE_K)
                        band_solve(c, q.vals, P->n_v, P->bwK, out->z3 + off3[i], R2, in->r2, 2);
                    else
                        band_solve(c, P->Lp_band.p, P->n_p, P->bwL, out->z3 + off3[i], R2, in->r2, 1);
                    break;
                }
                case S_EMBED_F:
                case S_EMBED_D: {
                    // rows of other blocks are written by their own launches; zero this block's rows first
                    copy_mat(c, n_x, in->r2, MatView{out->z3 + off3[i], R2, 1}, MatViewMut{out->z3 + off3[i], R2, 1}, 0.0);
                    const int nin = q.kind == S_EMBED_F ? P->n_v : P->n_D;
                    const int* map = q.kind == S_EMBED_F ? P->free_nodes.p : P->dir_nodes.p;
                    k_embed<<<std::min(4096, ceil_div(2LL * nin * in->r2, 256)), 256, 0, c->stream>>>(
                        nin, P->n_nodes, in->r2, map, in->z3, out->z3, R2, off3[i]);
                    LAUNCH_CHECK(c);
                    break;
                }
                default:
                    TT_THROW(TT_EINVAL, "unhandled spatial operator %d", (int)q.kind);
            }
        }
    }
    return out;
}

TTPtr apply_space(tt_ctx* c, tt_problem* P, const tt_t* in, SKind kind, double coef, const double* vals) {
    return kron_sum(c, P, {C1{in, T_COPY, nullptr}}, {C3{in, kind, vals, coef}}, {C2{0, 0, nullptr, 1.0, nullptr}});
}

// ============================================================== right-hand side
void make_rhs(tt_ctx* c, tt_problem* P) {
    const double ti = 1.0 / P->tau;
    const int m1 = P->m + 1;
    const size_t nnzD = std::max(1, P->fD.nnz), nxi2 = (size_t)P->n_xi * P->n_xi;
    if (!P->uD) {
        // no Dirichlet data: zero right-hand side
        P->fu = zeros(c, P->n_t, P->n_xi, 2 * P->n_v).release();
        P->fp = zeros(c, P->n_t, P->n_xi, P->n_p).release();
        P->fnorm = 0.0;
        return;
    }
    const tt_t* uD = P->uD;
    // f^u = -[tau^-1 (I - C) (x) I (x) M_fD + sum_l I (x) G_l (x) A_l,fD] u_D
    std::vector<C1> b1 = {C1{uD, T_COPY, nullptr}, C1{uD, T_SHIFT, nullptr}};
    std::vector<C3> b3 = {C3{uD, S_VELD, P->M_fD.p, 1.0}};
    for (int l = 0; l < m1; ++l) b3.push_back(C3{uD, S_VELD, P->A_fD.p + (size_t)l * nnzD, 1.0});
    std::vector<C2> b2 = {C2{0, 0, nullptr, -ti, nullptr}, C2{1, 0, nullptr, ti, nullptr}};
    for (int l = 0; l < m1; ++l) b2.push_back(C2{0, 1 + l, l == 0 ? nullptr : P->G.p + l * nxi2, -1.0, nullptr});
    P->fu = kron_sum(c, P, b1, b3, b2).release();
    P->fp = kron_sum(c, P, {C1{uD, T_COPY, nullptr}}, {C3{uD, S_DIVD, nullptr, -1.0}},
                     {C2{0, 0, nullptr, 1.0, nullptr}}).release();
    RoundOut a, b;
    round_tt(c, P->fu, 0.0, &a);
    round_tt(c, P->fp, 0.0, &b);
    P->fnorm = std::hypot(a.nrm_before, b.nrm_before);
}

TTPtr full_velocity(tt_ctx* c, tt_problem* P, const tt_t* u) {
    if (!P->uD)
        return kron_sum(c, P, {C1{u, T_COPY, nullptr}}, {C3{u, S_EMBED_F, nullptr, 1.0}}, {C2{0, 0, nullptr, 1.0, nullptr}});
    return kron_sum(c, P, {C1{u, T_COPY, nullptr}, C1{P->uD, T_COPY, nullptr}},
                    {C3{u, S_EMBED_F, nullptr, 1.0}, C3{P->uD, S_EMBED_D, nullptr, 1.0}},
                    {C2{0, 0, nullptr, 1.0, nullptr}, C2{1, 1, nullptr, 1.0, nullptr}});
}

// ============================================================== operators
namespace {
// wt[(a * kw2 + b) * n_xi + l] = w2[(a * n_xi + l) * kw2 + b]
__global__ void k_w2_perm(int kw1, int n_xi, int kw2, const double* __restrict__ w2, double* __restrict__ wt) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kw1 * n_xi * kw2) return;
    const int b = e % kw2, al = e / kw2, l = al % n_xi, a = al / n_xi;
    wt[((size_t)a * kw2 + b) * n_xi + l] = w2[e];
}
// w_avg(node) = sum_b cbar_b w3[node][b], cbar_b = mean_t cmean(t, b)
__global__ void k_wavg(int rows, int kw2, int n_t, const double* __restrict__ cm, const double* __restrict__ w3,
                       double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    double s = 0.0;
    for (int b = 0; b < kw2; ++b) {
        double cb = 0.0;
        for (int t = 0; t < n_t; ++t) cb += cm[(size_t)b * n_t + t];
        s += (cb / n_t) * w3[(size_t)i * kw2 + b];
    }
    out[i] = s;
}
}  // namespace

// convection data of an operator: N(w3_b) values, Hmix and the mean coefficients
static void conv_setup(tt_ctx* c, tt_op* op, bool need_hmix) {
    tt_problem* P = op->P;
    const tt_t* w = op->w.get();
    op->kw1 = w->r1;
    op->kw2 = w->r2;
    const int nnz = P->ff.nnz;
    op->Nff.alloc(c, (size_t)op->kw2 * nnz);
    assemble_conv(c, P, w->z3, w->r2, w->r2, op->Nff.p, nullptr);
    // c_b(t) = sum_a w1(t, a) w2(a, 0, b): n_t x kw2 column-major
    op->cmean.alloc(c, (size_t)P->n_t * op->kw2);
    gemm(c, P->n_t, op->kw2, op->kw1, 1.0, colmaj(w->z1, P->n_t), MatView{w->z2, (long long)P->n_xi * op->kw2, 1}, 0.0,
         colmaj(op->cmean.p, P->n_t));
    if (need_hmix) {
        const int n_xi = P->n_xi, q = op->kw1 * op->kw2;
        DBuf<double> wt(c, (size_t)q * n_xi);
        k_w2_perm<<<ceil_div((long long)q * n_xi, 256), 256, 0, c->stream>>>(op->kw1, n_xi, op->kw2, w->z2, wt.p);
        LAUNCH_CHECK(c);
        op->Hmix.alloc(c, (size_t)q * n_xi * n_xi);
        gemm(c, q, n_xi * n_xi, n_xi, 1.0, rowmaj(wt.p, n_xi), rowmaj(P->H.p, (long long)n_xi * n_xi), 0.0,
             rowmaj(op->Hmix.p, (long long)n_xi * n_xi));
    }
}

void op_init(tt_ctx* c, tt_op* op, tt_problem* P, const tt_t* w, int which) {
    op->P = P;
    op->which = which;
    if (w) {
        TT_REQUIRE(w->n_x == 2 * P->n_nodes && w->n_t == P->n_t && w->n_xi == P->n_xi,
                   "convection train must be a full-node velocity field");
        op->w = clone(c, w);
        conv_setup(c, op, which == TT_OP_FULL);
    }
}

bool op_wavg(tt_ctx* c, const tt_op* op, double* out) {
    tt_problem* P = op->P;
    if (!op->w) {
        fill_zero(c, out, 2 * (size_t)P->n_nodes);
        return false;
    }
    k_wavg<<<ceil_div(2 * P->n_nodes, 256), 256, 0, c->stream>>>(2 * P->n_nodes, op->kw2, P->n_t, op->cmean.p,
                                                                  op->w->z3, out);
    LAUNCH_CHECK(c);
    return true;
}

void op_ensure_K(tt_ctx* c, tt_op* op) {
    if (op->kready) return;
    tt_problem* P = op->P;
    op->Kband.alloc(c, (size_t)P->n_v * (2 * P->bwK + 1));
    if (op->w) {
        DBuf<double> wavg(c, 2 * (size_t)P->n_nodes);
        op_wavg(c, op, wavg.p);
        assemble_K_band(c, P, wavg.p, op->Kband.p);
    } else {
        assemble_K_band(c, P, nullptr, op->Kband.p);
    }
    op->kready = true;
}

void op_apply(tt_ctx* c, const tt_op* op, const tt_t* u, const tt_t* p, TTPtr* ou, TTPtr* op_) {
    tt_problem* P = op->P;
    TT_REQUIRE(op->which == TT_OP_FULL, "op_apply needs a FULL operator");
    TT_REQUIRE(u->n_x == 2 * P->n_v && p->n_x == P->n_p, "matvec: (u, p) sizes do not match the problem");
    const double ti = 1.0 / P->tau;
    const int m1 = P->m + 1;
    const size_t nnz = P->ff.nnz, nxi2 = (size_t)P->n_xi * P->n_xi;
    // u-output: tau^-1 (I-C) (x) I (x) M  +  sum_l I (x) G_l (x) A_l  +  N(w)  +  B^T p
    std::vector<C1> b1 = {C1{u, T_COPY, nullptr}, C1{u, T_SHIFT, nullptr}};
    std::vector<C3> b3 = {C3{u, S_VEL, P->M_ff.p, 1.0}};
    std::vector<C2> b2 = {C2{0, 0, nullptr, ti, nullptr}, C2{1, 0, nullptr, -ti, nullptr}};
    for (int l = 0; l < m1; ++l) {
        b3.push_back(C3{u, S_VEL, P->A_ff.p + l * nnz, 1.0});
        b2.push_back(C2{0, (int)b3.size() - 1, l == 0 ? nullptr : P->G.p + l * nxi2, 1.0, nullptr});
    }
    if (op->w) {
        const int base1 = (int)b1.size(), base3 = (int)b3.size();
        for (int a = 0; a < op->kw1; ++a) b1.push_back(C1{u, T_DIAG, op->w->z1 + (size_t)a * P->n_t});
        for (int b = 0; b < op->kw2; ++b) b3.push_back(C3{u, S_VEL, op->Nff.p + b * nnz, 1.0});
        for (int a = 0; a < op->kw1; ++a)
            for (int b = 0; b < op->kw2; ++b)
                b2.push_back(C2{base1 + a, base3 + b, op->Hmix.p + ((size_t)a * op->kw2 + b) * nxi2, 1.0, nullptr});
    }
    b1.push_back(C1{p, T_COPY, nullptr});
    b3.push_back(C3{p, S_GRAD, nullptr, 1.0});
    b2.push_back(C2{(int)b1.size() - 1, (int)b3.size() - 1, nullptr, 1.0, nullptr});
    *ou = kron_sum(c, P, b1, b3, b2);
    // p-output: (I (x) I (x) B) u
    *op_ = kron_sum(c, P, {C1{u, T_COPY, nullptr}}, {C3{u, S_DIV, nullptr, 1.0}}, {C2{0, 0, nullptr, 1.0, nullptr}});
}

void op_apply_mean(tt_ctx* c, const tt_op* op, const tt_t* u, TTPtr* ou) {
    tt_problem* P = op->P;
    TT_REQUIRE(u->n_x == 2 * P->n_v, "mean matvec: u size does not match the problem");
    const double ti = 1.0 / P->tau;
    // tau^-1 (I - C) (x) I (x) M + I (x) I (x) A_0 + N_0(w), with
    // N_0(w) = sum_b diag(c_b) (x) I (x) N(w3_b), c_b(t) = sum_a w1(t,a) w2(a,0,b)
    std::vector<C1> b1 = {C1{u, T_COPY, nullptr}, C1{u, T_SHIFT, nullptr}};
    std::vector<C3> b3 = {C3{u, S_VEL, P->M_ff.p, 1.0}, C3{u, S_VEL, P->A_ff.p, 1.0}};
    std::vector<C2> b2 = {C2{0, 0, nullptr, ti, nullptr}, C2{1, 0, nullptr, -ti, nullptr}, C2{0, 1, nullptr, 1.0, nullptr}};
    if (op->w) {
        const size_t nnz = P->ff.nnz;
        for (int b = 0; b < op->kw2; ++b) {
            b1.push_back(C1{u, T_DIAG, op->cmean.p + (size_t)b * P->n_t});
            b3.push_back(C3{u, S_VEL, op->Nff.p + b * nnz, 1.0});
            b2.push_back(C2{(int)b1.size() - 1, (int)b3.size() - 1, nullptr, 1.0, nullptr});
        }
    }
    *ou = kron_sum(c, P, b1, b3, b2);
}

void op_apply_mean_p(tt_ctx* c, tt_op* op, const tt_t* p, TTPtr* out) {
    tt_problem* P = op->P;
    TT_REQUIRE(p->n_x == P->n_p, "pressure mean matvec: p size does not match the problem");
    const double ti = 1.0 / P->tau;
    if (op->w && !op->pready) {
        // N_p(w3_b) for the columns of the convection field's last core
        const size_t nnz = std::max(1, P->pp.nnz);
        op->Npp.alloc(c, (size_t)op->kw2 * nnz);
        assemble_pconv(c, P, op->w->z3, op->kw2, op->kw2, op->Npp.p);
        op->pready = true;
    }
    // tau^-1 (I - C) (x) I (x) M_p + I (x) I (x) A_p,0 + N_p,0(w), with
    // N_p,0(w) = sum_b diag(c_b) (x) I (x) N_p(w3_b), c_b(t) = sum_a w1(t,a) w2(a,0,b)
    std::vector<C1> b1 = {C1{p, T_COPY, nullptr}, C1{p, T_SHIFT, nullptr}};
    std::vector<C3> b3 = {C3{p, S_PRES, P->Mp_pp.p, 1.0}, C3{p, S_PRES, P->Ap_pp.p, 1.0}};
    std::vector<C2> b2 = {C2{0, 0, nullptr, ti, nullptr}, C2{1, 0, nullptr, -ti, nullptr}, C2{0, 1, nullptr, 1.0, nullptr}};
    if (op->w) {
        const size_t nnz = std::max(1, P->pp.nnz);
        for (int b = 0; b < op->kw2; ++b) {
            b1.push_back(C1{p, T_DIAG, op->cmean.p + (size_t)b * P->n_t});
            b3.push_back(C3{p, S_PRES, op->Npp.p + b * nnz, 1.0});
            b2.push_back(C2{(int)b1.size() - 1, (int)b3.size() - 1, nullptr, 1.0, nullptr});
        }
    }
    *out = kron_sum(c, P, b1, b3, b2);
}

// ============================================================== residual
double residual(tt_ctx* c, tt_problem* P, const tt_t* u, const tt_t* p, double eps, TTPtr* ru, TTPtr* rp) {
    PrecScope fp64(c, 0);   // the Picard residual is FP64 in every precision mode
    RandScope exact(c, false);   // and its truncation deterministic
    const double ti = 1.0 / P->tau;
    const int m1 = P->m + 1;
    const size_t nnz = P->ff.nnz, nnzD = std::max(1, P->fD.nnz), nxi2 = (size_t)P->n_xi * P->n_xi;
    TTPtr w = full_velocity(c, P, u);          // untruncated convection field (Section 4.3)
    const int kw1 = w->r1, kw2 = w->r2;
    DBuf<double> Nff(c, (size_t)kw2 * nnz), NfD(c, (size_t)kw2 * nnzD);
    assemble_conv(c, P, w->z3, kw2, kw2, Nff.p, P->fD.nnz ? NfD.p : nullptr);
    DBuf<double> wt(c, (size_t)kw1 * kw2 * P->n_xi), Hmix(c, (size_t)kw1 * kw2 * nxi2);
    {
        const int q = kw1 * kw2, n_xi = P->n_xi;
        k_w2_perm<<<ceil_div((long long)q * n_xi, 256), 256, 0, c->stream>>>(kw1, n_xi, kw2, w->z2, wt.p);
        LAUNCH_CHECK(c);
        gemm(c, q, n_xi * n_xi, n_xi, 1.0, rowmaj(wt.p, n_xi), rowmaj(P->H.p, (long long)n_xi * n_xi), 0.0,
             rowmaj(Hmix.p, (long long)n_xi * n_xi));
    }
    // r_u = f_u - [linear part] u - B^T p - N_ff(w) u - N_fD(w) u_D
    std::vector<C1> b1 = {C1{P->fu, T_COPY, nullptr}, C1{u, T_COPY, nullptr}, C1{u, T_SHIFT, nullptr}};
    std::vector<C3> b3 = {C3{P->fu, S_COPY, nullptr, 1.0}, C3{u, S_VEL, P->M_ff.p, 1.0}};
    std::vector<C2> b2 = {C2{0, 0, nullptr, 1.0, nullptr}, C2{1, 1, nullptr, -ti, nullptr}, C2{2, 1, nullptr, ti, nullptr}};
    for (int l = 0; l < m1; ++l) {
        b3.push_back(C3{u, S_VEL, P->A_ff.p + l * nnz, 1.0});
        b2.push_back(C2{1, (int)b3.size() - 1, l == 0 ? nullptr : P->G.p + l * nxi2, -1.0, nullptr});
    }
    const tt_t* ins[2] = {u, P->uD};
    for (int which = 0; which < 2; ++which) {
        const tt_t* in = ins[which];
        if (!in) continue;
        const int base1 = (int)b1.size(), base3 = (int)b3.size();
        for (int a = 0; a < kw1; ++a) b1.push_back(C1{in, T_DIAG, w->z1 + (size_t)a * P->n_t});
        for (int b = 0; b < kw2; ++b)
            b3.push_back(which == 0 ? C3{in, S_VEL, Nff.p + b * nnz, 1.0} : C3{in, S_VELD, NfD.p + b * nnzD, 1.0});
        for (int a = 0; a < kw1; ++a)
            for (int b = 0; b < kw2; ++b)
                b2.push_back(C2{base1 + a, base3 + b, Hmix.p + ((size_t)a * kw2 + b) * nxi2, -1.0, nullptr});
    }
    b1.push_back(C1{p, T_COPY, nullptr});
    b3.push_back(C3{p, S_GRAD, nullptr, 1.0});
    b2.push_back(C2{(int)b1.size() - 1, (int)b3.size() - 1, nullptr, -1.0, nullptr});
    TTPtr rawu = kron_sum(c, P, b1, b3, b2);
    TTPtr rawp = kron_sum(c, P, {C1{P->fp, T_COPY, nullptr}, C1{u, T_COPY, nullptr}},
                          {C3{P->fp, S_COPY, nullptr, 1.0}, C3{u, S_DIV, nullptr, 1.0}},
                          {C2{0, 0, nullptr, 1.0, nullptr}, C2{1, 1, nullptr, -1.0, nullptr}});
    RoundOut a, b;
    round_pair(c, rawu.get(), rawp.get(), eps, ru, rp, &a, &b);
    return std::hypot(a.nrm_after, b.nrm_after);
}

}  // namespace tt
