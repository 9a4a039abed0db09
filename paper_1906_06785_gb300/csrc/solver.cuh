// Low-rank flexible GMRES (Algorithm 4.2), the mean-based LSC preconditioner
// (eq. prec, eq. mean_lsc, eq. 11_prec) and truncated inexact Picard
// (Algorithm 3.1).
#pragma once
#include <functional>

#include "op.cuh"

namespace tt {

// A Krylov vector: a velocity train and, for the coupled system, a pressure train.
struct Vec {
    TTPtr u{nullptr, tt_free};
    TTPtr p{nullptr, tt_free};
};

struct GmresOut {
    int its = 0;
    double res0 = 0.0, res = 0.0, bnorm = 0.0;
    bool converged = false;
};

using VecOp = std::function<Vec(const Vec&)>;

// Algorithm 4.2 with z_0 = 0.  apply_L returns the untruncated product.
Vec gmres(tt_ctx* c, const VecOp& apply_L, const VecOp& apply_P, const Vec& b, double tol, double eps, int maxit,
          double bnorm, GmresOut* out);

// Mean-based block triangular preconditioner for a FULL operator (its w).  With a
// network, the inner solve first runs with the learned M^-1 and is redone with the
// exact M^-1 when it misses tol_inner.
struct LSCPrec {
    tt_ctx* c;
    tt_op* op;
    double eps, tol_inner;
    int maxit_inner;
    const tt_net* net = nullptr;
    bool pcd = false;       // Schur part from eq. (mean_pcd) instead of eq. (mean_lsc)
    int inner_its = 0;
    int fallbacks = 0;
    Vec apply(const Vec& v);
    TTPtr schur(const tt_t* ap);
    TTPtr schur_pcd(const tt_t* ap);
    TTPtr minv(const tt_t* z);
};

// M^-1 z of eq. (11_prec) with the network in place of K^-1 (learned.cu).
TTPtr learned_minv(tt_ctx* c, const tt_net* net, tt_op* op, const tt_t* z);

void picard(tt_ctx* c, tt_problem* P, const tt_solver_opts* o, TTPtr* u, TTPtr* p, tt_picard_stats* st);

}  // namespace tt
