// Device-resident discretisation of the all-at-once problem (Sections 3.2, 3.3,
// 5.1): CSR patterns, assembled Q2-Q1 matrices, gPC matrices, the Dirichlet
// lifting and the right-hand side, plus sparse and banded kernels.
#pragma once
#include "tt.cuh"

namespace tt {

struct Csr {
    int n_rows = 0, n_cols = 0, nnz = 0;
    DBuf<int> rowptr, col;
};
// For each CSR slot, the list of element-local entries summed into it.
struct Gather {
    DBuf<int> ptr, idx;
};

// Sparse kernels --------------------------------------------------------------
// Y[(c*n_rows + i)*ldy + coff[k] + b] = coef[k] * sum_nz vals[k][nz] X[(c*n_in + col)*ldx + b]
// for components c < ncomp (both velocity components, or one), k < nmat (<= 8), b < ncol.
struct VelSpmm {
    const int* rowptr;
    const int* col;
    int n_rows, n_in;
    int ncomp;          // components (2: velocity; 1: a scalar pressure-space matrix)
    int nnz;
    int nmat;
    const double* vals[8];
    double coef[8];
    int coff[8];
};
void spmm_vel(tt_ctx* c, const VelSpmm& s, const double* X, int ldx, double* Y, int ldy, int ncol);
// pressure rows: Y[i*ldy + coff + b] = coef sum_nz (Bx[nz] X[col] + By[nz] X[n_in + col])
void spmm_div(tt_ctx* c, const Csr& B, const double* Bx, const double* By, int n_in, double coef,
              const double* X, int ldx, double* Y, int ldy, int coff, int ncol);
// velocity rows (c, j): Y[(c*n_rows + j)*ldy + coff + b] = coef sum_nz BTc[nz] X[col*ldx + b]
void spmm_grad(tt_ctx* c, const Csr& BT, const double* BTx, const double* BTy, double coef,
               const double* X, int ldx, double* Y, int ldy, int coff, int ncol);

// Band matrices (no pivoting; row-major band, element (i, j) at i*(2bw+1) + j - i + bw)
void band_factor(tt_ctx* c, double* ab, int n, int bw);
// Solve (LU) x = b in place for ncol columns of X, rows (comp*n + i), comp < ncomp,
// element at (comp*n + i)*ldx + b.
void band_solve(tt_ctx* c, const double* ab, int n, int bw, double* X, int ldx, int ncol, int ncomp);

}  // namespace tt

struct tt_problem {
    tt_ctx* ctx = nullptr;
    int n_nodes = 0, n_elem = 0, n_p = 0, n_v = 0, n_D = 0, m = 0, n_xi = 0, n_t = 0;
    double tau = 0.0, h = 0.0;
    std::vector<int> fidx, didx;            // node -> free / Dirichlet index or -1
    std::vector<double> hxy;                // node coordinates (host copy, n_nodes x 2)
    tt::DBuf<int> eq2, eq1;                 // element connectivity
    tt::DBuf<int> node_free, node_dir;      // device copies of fidx / didx
    tt::DBuf<int> free_nodes, dir_nodes;    // free / Dirichlet index -> node
    tt::Csr ff, fD, BF, BD, BT, pp;         // patterns (pp: Q1 pressure space)
    tt::Gather g_ff, g_fD, g_BF, g_BD, g_pp;  // assembly gather maps
    tt::DBuf<int> bt_perm;                  // BT slot -> BF slot
    tt::DBuf<int> diag_slot;                // ff slot of (i, i)
    tt::DBuf<double> nu;                    // (m+1) x n_p nodal viscosities
    tt::DBuf<double> M_ff, M_fD;            // scalar mass
    tt::DBuf<double> A_ff, A_fD;            // (m+1) x nnz
    tt::DBuf<double> Bx_F, By_F, Bx_D, By_D, BTx, BTy;
    tt::DBuf<double> Mstar;                 // diag of M_ff (n_v)
    tt::DBuf<int> pdiag_slot;               // pp slot of (i, i)
    tt::DBuf<double> Mp_pp, Ap_pp;          // pressure mass, mean pressure diffusion (pp)
    tt::DBuf<double> Mpstar;                // diag of M_p (n_p)
    tt::DBuf<double> G;                     // (m+1) x n_xi x n_xi
    tt::DBuf<double> H;                     // n_xi x n_xi x n_xi  H[l][r][s]
    std::vector<double> hG;                 // host copy of G
    int bwK = 0, bwL = 0;                   // half bandwidths of K (ff) and L_p
    tt::DBuf<double> Lp_band;               // factorised B M*^-1 B^T
    tt_t* uD = nullptr;                     // lifting (rank 1, 2 n_D rows)
    tt_t* fu = nullptr;                     // right-hand side
    tt_t* fp = nullptr;
    double fnorm = 0.0;
    ~tt_problem();
};

namespace tt {
// Local element matrices and assembly (fem.cu)
// Convection N(w) values on the ff (and optionally fD) pattern for nf fields
// w_k(node) = (W[(node)*ldw + col_k], W[(n_nodes + node)*ldw + col_k]) with col_k = k.
void assemble_conv(tt_ctx* c, tt_problem* P, const double* W, int ldw, int nf, double* vals_ff,
                   double* vals_fD);
// Pressure-space convection N_p(w) values on the pp pattern for nf fields (as above)
void assemble_pconv(tt_ctx* c, tt_problem* P, const double* W, int ldw, int nf, double* vals_pp);
// Values of K = tau^-1 M + A_0 + N(w) on the ff pattern (w full-node field or null)
void assemble_K_vals(tt_ctx* c, tt_problem* P, const double* wfield, double* kv);
// K = tau^-1 M + A_0 + N(w) scattered into band storage and factorised (LU)
void assemble_K_band(tt_ctx* c, tt_problem* P, const double* wfield, double* ab);
// Scatter ff-pattern values into band storage
void scatter_band(tt_ctx* c, tt_problem* P, const double* vals, double* ab);
void build_problem(tt_ctx* c, tt_problem* P, const tt_problem_desc* d);
}  // namespace tt
