// Kronecker-structured operators of the all-at-once system (eq. F, eq. N_kron,
// Section 5.2) applied to trains, and the mean-based preconditioner (Section 5).
#pragma once
#include "problem.cuh"

namespace tt {

// ---- generic sum of Kronecker terms  sum_k (T_k (x) S_k (x) F_k) in_k ----------
enum TKind { T_COPY, T_SHIFT, T_DIAG, T_CUMSUM };
enum SKind {
    S_COPY,      // identity
    S_VEL,       // scalar ff matrix on both velocity components (vals on P->ff)
    S_VELD,      // scalar fD matrix: 2 n_D rows in, n_u rows out (vals on P->fD)
    S_DIV,       // B over free dofs: n_u -> n_p
    S_DIVD,      // B over Dirichlet dofs: 2 n_D -> n_p
    S_GRAD,      // B^T: n_p -> n_u
    S_MSTARINV,  // M_*^{-1} on both components
    S_SOLVE_K,   // banded K^{-1} on both components (band = factor)
    S_SOLVE_LP,  // banded L_p^{-1} (problem's factor)
    S_EMBED_F,   // free velocity dofs -> full-node field (2 n_nodes rows)
    S_EMBED_D,   // Dirichlet dofs -> full-node field
    S_PRES,      // scalar pressure-space matrix (vals on P->pp): n_p -> n_p
    S_MPSTARINV  // M_p*^{-1} = diag(M_p)^{-1} on a pressure train
};
struct C1 {            // core-1 block: time operator on an input's first core
    const tt_t* in;
    TKind kind;
    const double* vec;  // T_DIAG: n_t values
};
struct C3 {            // core-3 block: spatial operator on an input's last core
    const tt_t* in;
    SKind kind;
    const double* vals;   // S_VEL / S_VELD values, or S_SOLVE_K band
    double coef;
};
struct C2 {            // core-2 block at (c1 block, c3 block): coef * dcoef * S (x) on middle core
    int b1, b3;
    const double* S;      // n_xi x n_xi row-major on device, nullptr = identity
    double coef;
    const double* dcoef;  // device scalar or nullptr
};
TTPtr kron_sum(tt_ctx* c, tt_problem* P, const std::vector<C1>& b1, const std::vector<C3>& b3,
               const std::vector<C2>& b2);

// single spatial operator applied to a train (cores 1, 2 copied)
TTPtr apply_space(tt_ctx* c, tt_problem* P, const tt_t* in, SKind kind, double coef = 1.0,
                  const double* vals = nullptr);

// right-hand side and lifting
void make_rhs(tt_ctx* c, tt_problem* P);
TTPtr full_velocity(tt_ctx* c, tt_problem* P, const tt_t* u);
// residual r = f - A(w)[u; p] (w = E u + u_D), truncated; returns ||T(r)||
double residual(tt_ctx* c, tt_problem* P, const tt_t* u, const tt_t* p, double eps, TTPtr* ru, TTPtr* rp);

}  // namespace tt

struct tt_op {
    tt_problem* P = nullptr;
    int which = TT_OP_FULL;
    tt::TTPtr w{nullptr, tt::tt_free};     // convection train (full-node), may be null
    int kw1 = 0, kw2 = 0;
    tt::DBuf<double> Nff;     // kw2 x nnz(ff): N(w3_b)
    tt::DBuf<double> Hmix;    // kw1 x kw2 x n_xi x n_xi (FULL)
    tt::DBuf<double> cmean;   // n_t x kw2, column-major: c_b(t) = sum_a w1(t,a) w2(a,0,b)
    tt::DBuf<double> Kband;   // factorised tau^-1 M + A_0 + N(w_avg)
    bool kready = false;
    tt::DBuf<double> Npp;     // kw2 x nnz(pp): N_p(w3_b) on the pressure space (PCD)
    bool pready = false;
};

namespace tt {
void op_init(tt_ctx* c, tt_op* op, tt_problem* P, const tt_t* w, int which);
// L[u; p] (FULL) or (F_0 + C) u (MEAN) without truncation
void op_apply(tt_ctx* c, const tt_op* op, const tt_t* u, const tt_t* p, TTPtr* ou, TTPtr* op_);
void op_apply_mean(tt_ctx* c, const tt_op* op, const tt_t* u, TTPtr* ou);
// (F_p,0 + C_p) p on the pressure space (Section 5.2) without truncation
void op_apply_mean_p(tt_ctx* c, tt_op* op, const tt_t* p, TTPtr* out);
void op_ensure_K(tt_ctx* c, tt_op* op);
// w_avg of eq. (11_prec) (full-node, 2 n_nodes values) into out; zeros and false
// when the operator has no convection field
bool op_wavg(tt_ctx* c, const tt_op* op, double* out);
}  // namespace tt
