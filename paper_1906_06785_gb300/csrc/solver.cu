// Solvers: Algorithm 4.2 (low-rank flexible GMRES), the mean-based LSC
// preconditioner of Section 5 and the truncated inexact Picard iteration of
// Algorithm 3.1.  Fixed choices where the paper leaves room: z_0 = 0, no
// restarts, modified Gram-Schmidt coefficients h_ik = <x - sum_{j<i} h_jk v_j, v_i>
// (evaluated from <x, v_i> and the basis Gram matrix), h_{k+1,k} = ||x|| from the
// orthogonalised train with v_{k+1} = T(x) / h_{k+1,k}, stopping on the norm of
// the truncated s_k, happy breakdown when h_{k+1,k} <= 1e-14 beta.  The
// Hessenberg least-squares problem is solved on the device in FP64 (Givens).
#include <algorithm>
#include <cmath>

#include "solver.cuh"

namespace tt {

namespace {
__global__ void k_set(double* p, double v) { *p = v; }
__global__ void k_add_to(double* dst, const double* a, const double* b) { *dst = *a + *b; }

// h_i = d_i - sum_{j<i} h_j G[j][i]  (modified Gram-Schmidt via the basis Gram matrix)
__global__ void k_mgs(int k, const double* __restrict__ d, const double* __restrict__ G, int ldg, double* __restrict__ h) {
    if (threadIdx.x || blockIdx.x) return;
    for (int i = 0; i < k; ++i) {
        double s = d[i];
        for (int j = 0; j < i; ++j) s -= h[j] * G[(size_t)i * ldg + j];
        h[i] = s;
    }
}

// y = argmin || beta e_1 - Hbar y ||, Hbar (k+1) x k column-major with leading dim ldh (Givens QR)
__global__ void k_lsq(int k, const double* __restrict__ Hbar, int ldh, double beta, double* __restrict__ y) {
    if (threadIdx.x || blockIdx.x) return;
    double R[64][64];
    double g[65];
    const int kk = k;
    for (int j = 0; j < kk; ++j)
        for (int i = 0; i <= kk; ++i) R[i][j] = 0.0;
    for (int j = 0; j < kk; ++j)
        for (int i = 0; i <= j + 1; ++i) R[i][j] = Hbar[(size_t)j * ldh + i];
    for (int i = 0; i <= kk; ++i) g[i] = 0.0;
    g[0] = beta;
    for (int j = 0; j < kk; ++j) {
        const double a = R[j][j], b = R[j + 1][j];
        const double r = hypot(a, b);
        const double cs = r == 0.0 ? 1.0 : a / r, sn = r == 0.0 ? 0.0 : b / r;
        for (int l = j; l < kk; ++l) {
            const double x = R[j][l], z = R[j + 1][l];
            R[j][l] = cs * x + sn * z;
            R[j + 1][l] = -sn * x + cs * z;
        }
        const double x = g[j], z = g[j + 1];
        g[j] = cs * x + sn * z;
        g[j + 1] = -sn * x + cs * z;
    }
    for (int i = kk - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < kk; ++l) s -= R[i][l] * y[l];
        y[i] = R[i][i] != 0.0 ? s / R[i][i] : 0.0;
    }
}
}  // namespace

// ---------------------------------------------------------------- vector helpers
static Vec vround(tt_ctx* c, const Vec& v, double eps, double* before, double* after) {
    Vec r;
    RoundOut a, b;
    if (v.p) round_pair(c, v.u.get(), v.p.get(), eps, &r.u, &r.p, &a, &b);
    else r.u = round_any(c, v.u.get(), eps, &a);
    if (before) *before = std::hypot(a.nrm_before, b.nrm_before);
    if (after) *after = std::hypot(a.nrm_after, b.nrm_after);
    return r;
}

struct VTerm {
    double coef;
    const double* dcoef;
    const Vec* v;
};
static Vec vcat(tt_ctx* c, const std::vector<VTerm>& terms) {
    Vec r;
    std::vector<Summand> su, sp;
    for (auto& t : terms) {
        su.push_back(Summand{t.coef, t.dcoef, t.v->u.get()});
        if (t.v->p) sp.push_back(Summand{t.coef, t.dcoef, t.v->p.get()});
    }
    r.u = concat(c, su);
    if (!sp.empty()) r.p = concat(c, sp);
    return r;
}

static Vec vscale(tt_ctx* c, const Vec& v, double s) {
    Vec r;
    r.u = clone(c, v.u.get(), s);
    if (v.p) r.p = clone(c, v.p.get(), s);
    return r;
}

static void vdot(tt_ctx* c, const Vec& a, const Vec& b, double* dout, double* tmp2) {
    if (!a.p) {
        dot_dev(c, a.u.get(), b.u.get(), dout);
        return;
    }
    dot_dev(c, a.u.get(), b.u.get(), tmp2);
    dot_dev(c, a.p.get(), b.p.get(), tmp2 + 1);
    k_add_to<<<1, 1, 0, c->stream>>>(dout, tmp2, tmp2 + 1);
    LAUNCH_CHECK(c);
}

static Vec vzeros_like(tt_ctx* c, const Vec& b) {
    Vec r;
    r.u = zeros(c, b.u->n_t, b.u->n_xi, b.u->n_x);
    if (b.p) r.p = zeros(c, b.p->n_t, b.p->n_xi, b.p->n_x);
    return r;
}

// ---------------------------------------------------------------- Algorithm 4.2
Vec gmres(tt_ctx* c, const VecOp& apply_L, const VecOp& apply_P, const Vec& b, double tol, double eps, int maxit,
          double bnorm, GmresOut* out) {
    TT_REQUIRE(maxit >= 1 && maxit <= 63, "maxit must be in [1, 63]");
    double before = 0.0, beta = 0.0;
    Vec s0 = vround(c, b, eps, &before, &beta);      // s_0 = T(b - L 0)
    if (bnorm <= 0.0) bnorm = before;
    out->bnorm = bnorm;
    out->res0 = beta;
    out->res = beta;
    out->its = 0;
    out->converged = beta <= tol * bnorm;
    if (beta == 0.0 || out->converged) return vzeros_like(c, b);
    const int ld = maxit + 1;
    DBuf<double> dH(c, (size_t)ld * maxit), dG(c, (size_t)ld * ld), dd(c, ld), dy(c, maxit), tmp(c, 2);
    fill_zero(c, dH.p, (size_t)ld * maxit);
    std::vector<Vec> V, Vh;
    V.push_back(vscale(c, s0, 1.0 / beta));
    Vec z;
    double res = beta;
    int k = 0;
    while (res > tol * bnorm && k < maxit) {
        ++k;
        Vh.push_back(apply_P(V[k - 1]));
        Vec x = vround(c, apply_L(Vh[k - 1]), eps, nullptr, nullptr);
        for (int i = 0; i < k; ++i) vdot(c, x, V[i], dd.p + i, tmp.p);
        double* hcol = dH.p + (size_t)(k - 1) * ld;
        k_mgs<<<1, 1, 0, c->stream>>>(k, dd.p, dG.p, ld, hcol);
        LAUNCH_CHECK(c);
        std::vector<VTerm> terms = {VTerm{1.0, nullptr, &x}};
        for (int i = 0; i < k; ++i) terms.push_back(VTerm{-1.0, hcol + i, &V[i]});
        double hk = 0.0;
        Vec xr = vround(c, vcat(c, terms), eps, &hk, nullptr);     // h_{k+1,k} = ||x||
        k_set<<<1, 1, 0, c->stream>>>(hcol + k, hk);
        LAUNCH_CHECK(c);
        const bool breakdown = hk <= 1e-14 * beta;
        if (!breakdown) {
            V.push_back(vscale(c, xr, 1.0 / hk));
            for (int j = 0; j < k; ++j) vdot(c, V[j], V[k], dG.p + (size_t)k * ld + j, tmp.p);
        }
        k_lsq<<<1, 1, 0, c->stream>>>(k, dH.p, ld, beta, dy.p);
        LAUNCH_CHECK(c);
        std::vector<VTerm> zt;
        for (int i = 0; i < k; ++i) zt.push_back(VTerm{1.0, dy.p + i, &Vh[i]});
        z = vround(c, vcat(c, zt), eps, nullptr, nullptr);
        Vec Lz = apply_L(z);
        vround(c, vcat(c, {VTerm{1.0, nullptr, &b}, VTerm{-1.0, nullptr, &Lz}}), eps, nullptr, &res);
        if (breakdown) break;
    }
    out->its = k;
    out->res = res;
    out->converged = res <= tol * bnorm;
    return z;
}

// ---------------------------------------------------------------- preconditioner
TTPtr LSCPrec::minv(const tt_t* z) {
    op_ensure_K(c, op);
    return kron_sum(c, op->P, {C1{z, T_CUMSUM, nullptr}}, {C3{z, S_SOLVE_K, op->Kband.p, 1.0}},
                    {C2{0, 0, nullptr, 1.0, nullptr}});
}

TTPtr LSCPrec::schur_pcd(const tt_t* ap) {
    // p = -L^-1 (F_p,0 + C_p) M_p*^-1 a_p  (eq. mean_pcd), L = B M*^-1 B^T
    tt_problem* P = op->P;
    TTPtr y = apply_space(c, P, ap, S_MPSTARINV);
    TTPtr fy{nullptr, tt_free};
    op_apply_mean_p(c, op, y.get(), &fy);
    y = round_any(c, fy.get(), eps);
    return apply_space(c, P, y.get(), S_SOLVE_LP, -1.0);
}

TTPtr LSCPrec::schur(const tt_t* ap) {
    if (pcd) return schur_pcd(ap);
    // p = -L^-1 (B M*^-1 (F_0 + C) M*^-1 B^T) L^-1 a_p  (eq. mean_lsc), L = B M*^-1 B^T
    tt_problem* P = op->P;
    TTPtr y = apply_space(c, P, ap, S_SOLVE_LP);
    y = apply_space(c, P, y.get(), S_GRAD);
    y = apply_space(c, P, y.get(), S_MSTARINV);
    TTPtr my{nullptr, tt_free};
    op_apply_mean(c, op, y.get(), &my);
    y = round_any(c, my.get(), eps);
    y = apply_space(c, P, y.get(), S_MSTARINV);
    y = apply_space(c, P, y.get(), S_DIV);
    return apply_space(c, P, y.get(), S_SOLVE_LP, -1.0);
}

Vec LSCPrec::apply(const Vec& v) {
    tt_problem* P = op->P;
    Vec r;
    r.p = schur(v.p.get());
    TTPtr bt = apply_space(c, P, r.p.get(), S_GRAD);
    TTPtr rhs = round_any(c, concat(c, {Summand{1.0, nullptr, v.u.get()}, Summand{-1.0, nullptr, bt.get()}}).get(), eps);
    // (F_0 + C) u = rhs by inner low-rank GMRES preconditioned with M (Section 5.3)
    Vec b;
    b.u = std::move(rhs);
    GmresOut go;
    tt_op* o = op;
    tt_ctx* cc = c;
    const VecOp apply_mean = [o, cc](const Vec& x) { Vec y; op_apply_mean(cc, o, x.u.get(), &y.u); return y; };
    if (net) {
        // the learned attempt gets a fifth of the inner budget (at least 4 iterations):
        // a network that does not reach tol_inner by then hands over to the exact M^-1
        const tt_net* nn = net;
        const int maxit_learned = std::max(4, maxit_inner / 5);
        Vec u = gmres(
            c, apply_mean, [cc, nn, o](const Vec& x) { Vec y; y.u = learned_minv(cc, nn, o, x.u.get()); return y; },
            b, tol_inner, eps, std::min(maxit_inner, maxit_learned), 0.0, &go);
        inner_its += go.its;
        if (go.converged) {
            r.u = std::move(u.u);
            return r;
        }
        ++fallbacks;
    }
    Vec u = gmres(
        c, apply_mean, [this](const Vec& x) { Vec y; y.u = minv(x.u.get()); return y; },
        b, tol_inner, eps, maxit_inner, 0.0, &go);
    inner_its += go.its;
    r.u = std::move(u.u);
    return r;
}

// ---------------------------------------------------------------- Algorithm 3.1
static VecOp full_op(tt_ctx* c, tt_op* op) {
    return [c, op](const Vec& x) {
        Vec y;
        op_apply(c, op, x.u.get(), x.p.get(), &y.u, &y.p);
        return y;
    };
}

void picard(tt_ctx* c, tt_problem* P, const tt_solver_opts* o, TTPtr* uo, TTPtr* po, tt_picard_stats* st) {
    TT_REQUIRE(o, "null options");
    TT_REQUIRE(o->precision == TT_FP64 || o->precision == TT_MIXED, "unknown precision %d", o->precision);
    TT_REQUIRE(o->rounding == TT_ROUND_EXACT || o->rounding == TT_ROUND_RANDOMIZED, "unknown rounding %d",
               o->rounding);
    TT_REQUIRE((o->init_u == nullptr) == (o->init_p == nullptr), "init_u and init_p go together");
    TT_REQUIRE(o->schur == TT_PREC_LSC || o->schur == TT_PREC_PCD, "schur must be TT_PREC_LSC or TT_PREC_PCD");
    memset(st, 0, sizeof(*st));
    st->fnorm = P->fnorm;
    const int fast = o->precision == TT_MIXED ? 1 : 0;
    TTPtr u{nullptr, tt_free}, p{nullptr, tt_free};
    if (o->init_u) {
        // resume from a given iterate (Algorithm 3.1 from step i = 0 with u^(0), p^(0))
        TT_REQUIRE(o->init_u->n_x == 2 * P->n_v && o->init_p->n_x == P->n_p && o->init_u->n_t == P->n_t &&
                       o->init_u->n_xi == P->n_xi && o->init_p->n_t == P->n_t && o->init_p->n_xi == P->n_xi,
                   "initial iterate does not match the problem");
        u = clone(c, o->init_u);
        p = clone(c, o->init_p);
    } else {
        Vec f;
        f.u = clone(c, P->fu);
        f.p = clone(c, P->fp);
        // Stokes problem (N = 0) for the initial iterate, solved to tol_gmres ||f|| (Section 5.2)
        tt_op stokes;
        op_init(c, &stokes, P, nullptr, TT_OP_FULL);
        LSCPrec pre{c, &stokes, o->eps_gmres, o->tol_inner, o->maxit_inner, o->learned, o->schur == TT_PREC_PCD};
        GmresOut go;
        Vec up;
        {
            PrecScope ps(c, fast);
            RandScope rs(c, o->rounding == TT_ROUND_RANDOMIZED);
            up = gmres(c, full_op(c, &stokes), [&pre](const Vec& v) { return pre.apply(v); }, f, o->tol_gmres,
                       o->eps_gmres, o->maxit_gmres, P->fnorm, &go);
        }
        st->stokes_its = go.its;
        st->gmres_its[0] = go.its;
        st->inner_its[0] = pre.inner_its;
        st->fallbacks[0] = pre.fallbacks;
        u = std::move(up.u);
        p = std::move(up.p);
    }
    TTPtr ru{nullptr, tt_free}, rp{nullptr, tt_free};
    double rn = residual(c, P, u.get(), p.get(), o->eps_gmres, &ru, &rp);
    st->res[0] = rn;
    st->ranks[0][0] = u->r1; st->ranks[0][1] = u->r2; st->ranks[0][2] = p->r1; st->ranks[0][3] = p->r2;
    int i = 0;
    const int maxit = std::min(o->maxit_picard, TT_MAX_PICARD);
    while (rn > o->tol_picard * P->fnorm && i < maxit) {
        ++i;
        TTPtr w = full_velocity(c, P, u.get());
        TTPtr wt = round_tt(c, w.get(), o->eps_conv);                 // eq. (eps_conv)
        st->conv_ranks[i][0] = wt->r1; st->conv_ranks[i][1] = wt->r2;
        tt_op L;
        op_init(c, &L, P, wt.get(), TT_OP_FULL);
        LSCPrec pr{c, &L, o->eps_gmres, o->tol_inner, o->maxit_inner, o->learned, o->schur == TT_PREC_PCD};
        Vec r;
        r.u = std::move(ru);
        r.p = std::move(rp);
        Vec d;
        GmresOut go;
        {
            PrecScope ps(c, fast);
            RandScope rs(c, o->rounding == TT_ROUND_RANDOMIZED);
            d = gmres(c, full_op(c, &L), [&pr](const Vec& v) { return pr.apply(v); }, r, o->tol_gmres,
                      o->eps_gmres, o->maxit_gmres, rn, &go);
        }
        st->gmres_its[i] = go.its;
        st->inner_its[i] = pr.inner_its;
        st->fallbacks[i] = pr.fallbacks;
        u = round_tt(c, concat(c, {Summand{1.0, nullptr, u.get()}, Summand{1.0, nullptr, d.u.get()}}).get(), o->eps_soln);
        p = round_tt(c, concat(c, {Summand{1.0, nullptr, p.get()}, Summand{1.0, nullptr, d.p.get()}}).get(), o->eps_soln);
        rn = residual(c, P, u.get(), p.get(), o->eps_gmres, &ru, &rp);
        st->res[i] = rn;
        st->ranks[i][0] = u->r1; st->ranks[i][1] = u->r2; st->ranks[i][2] = p->r1; st->ranks[i][3] = p->r2;
    }
    st->picard_its = i;
    *uo = std::move(u);
    *po = std::move(p);
}

}  // namespace tt
