/*
 * tt_stochns.h -- C ABI of the GPU low-rank all-at-once solver for the
 * stochastic unsteady Navier-Stokes problem (Elman & Su, "A low-rank solver
 * for the stochastic unsteady Navier-Stokes problem").
 *
 * Conventions for every entry point:
 *   - returns an int status: TT_OK (0) or a negative TT_E* code; never throws;
 *     tt_last_error(ctx) gives a message for the last failure in that context;
 *   - all GPU work is enqueued on the context's CUDA stream; entry points that
 *     return host values (norms, ranks, statistics) synchronise that stream;
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     device memory of the current device; the flag arguments say which;
 *   - objects returned through out-parameters (tt_t, tt_problem, tt_op) are
 *     owned by the caller and released with their *_destroy function; the
 *     library copies every input array it keeps.
 *
 * Tensor-train layout (Section 4.1, eq. z_tt): a tensor z in
 * R^{n_t x n_xi x n_x} is z(i1,i2,i3) = sum z1(i1,a1) z2(a1,i2,a2) z3(a2,i3),
 * with cores passed and returned as
 *   z1: n_t x r1, column-major          (element (t,a)   at a*n_t + t)
 *   z2: r1 x n_xi x r2, r2 fastest      (element (a,s,b) at (a*n_xi + s)*r2 + b)
 *   z3: r2 x n_x, stored as n_x x r2 row-major (element (b,j) at j*r2 + b)
 * all in float64.  Velocity trains have n_x = n_u = 2 n_v (x1 components of
 * the free nodes first, then x2 components); pressure trains n_x = n_p;
 * full-node velocity fields (convection trains) n_x = 2 n_nodes.
 */
#ifndef TT_STOCHNS_H
#define TT_STOCHNS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    TT_OK = 0,
    TT_EINVAL = -1,      /* bad argument (shape, null pointer, mismatch) */
    TT_ENOMEM = -2,      /* device or host allocation failed */
    TT_ECUDA = -3,       /* a CUDA call failed (message in tt_last_error) */
    TT_ENOCONV = -4,     /* iteration cap reached; best iterate returned */
    TT_ERANK = -5,       /* a rank would exceed the configured capacity */
    TT_ENAN = -6,        /* non-finite value met in a norm */
    TT_ETIMEOUT = -7     /* a device-side wait ran out of its iteration budget */
};

typedef struct tt_ctx tt_ctx;
typedef struct tt_t tt_t;
typedef struct tt_problem tt_problem;
typedef struct tt_op tt_op;
typedef struct tt_prec tt_prec;
typedef struct tt_net tt_net;

/* Caller-supplied device allocator (for example a framework's caching allocator).
 * alloc returns `bytes` of device memory usable in stream order on `stream` (a
 * cudaStream_t), or NULL on failure (the call then fails with TT_ENOMEM); free
 * releases a block alloc returned, with the same size, in stream order.  `user`
 * is passed through unchanged.  The callbacks may be called from any thread that
 * calls into the library. */
typedef void* (*tt_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*tt_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* ---- context ------------------------------------------------------------ */

/* Create a context on the current CUDA device.  cuda_stream: a cudaStream_t
 * (NULL = the legacy default stream) on which all work of this context runs.
 * alloc, free: device memory for every train and every work buffer of this
 * context; both NULL = the library's own stream-ordered pool (cudaMallocAsync).
 * Passing only one of the two is TT_EINVAL.  A few bytes of bookkeeping (status
 * word, barrier counters, pinned staging) are allocated by the library itself. */
int tt_ctx_create(void* cuda_stream, tt_alloc_fn alloc, tt_free_fn free, void* user, tt_ctx** out);
int tt_ctx_destroy(tt_ctx* ctx);
/* Message of the last failure in this context (static storage, never NULL). */
const char* tt_last_error(const tt_ctx* ctx);
/* Number of kernels this context has launched so far. */
long long tt_ctx_launches(const tt_ctx* ctx);
/* Bound on device-side waits: a block of a cooperative (grid-synchronised) kernel
 * that has polled a grid barrier `polls` times gives up, records a timeout in the
 * context's device status word and finishes; the entry point then returns
 * TT_ETIMEOUT and clears the status word, and the context stays usable.  The
 * default (2e7 polls with back-off, seconds) never triggers in a healthy launch;
 * small values exist to exercise the failure path (0: any wait that cannot end at
 * once gives up).  polls < 0 is TT_EINVAL. */
int tt_ctx_set_wait_limit(tt_ctx* ctx, long long polls);

/* Profiling of kernel classes (0 QR, 1 Jacobi SVD, 2 GEMM, 3 SpMM, 4 banded
 * solve, 5 banded factorisation, 6 core-1/core-2/concatenation kernels,
 * 7 element assembly): CUDA events around each launch of a class on the
 * context stream, with the algorithmic flops and bytes of the launch.
 * tt_ctx_profile resets the counters and turns timing on (1) or off (0);
 * tt_ctx_prof_read synchronises the stream and returns the totals since the
 * last reset: launches, milliseconds, flops, bytes. */
int tt_ctx_profile(tt_ctx* ctx, int enable);
int tt_ctx_prof_read(tt_ctx* ctx, int slot, long long* launches, double* ms, double* flops,
                     double* bytes);

/* ---- tensor trains (Section 4.1) ------------------------------------------ */

enum { TT_F64 = 0 };   /* storage type of train cores (FP64 is the only one) */

/* Copy cores (layout above) into a new device-resident train of ranks (r1, r2)
 * whose allocation can hold ranks up to (rcap1, rcap2) (rcap <= 0: equal to the
 * rank; rcap < rank is TT_EINVAL).  dtype: TT_F64.
 * src_on_device: 0 = the three pointers are host memory, 1 = device memory. */
int tt_create(tt_ctx* ctx, int n_t, int n_xi, int n_x, int r1, int r2, int rcap1, int rcap2, int dtype,
              const double* z1, const double* z2, const double* z3, int src_on_device, tt_t** out);
int tt_destroy(tt_t* t);
int tt_shape(const tt_t* t, int* n_t, int* n_xi, int* n_x, int* r1, int* r2);
/* Rank capacities of the train's allocation. */
int tt_capacity(const tt_t* t, int* rcap1, int* rcap2);
/* Copy the cores out (buffers sized from tt_shape). */
int tt_get_cores(tt_ctx* ctx, const tt_t* t, double* z1, double* z2, double* z3,
                 int dst_on_device);

/* Truncation T_eps (Section 4.1): returns a train with
 * ||T(z) - z||_F <= eps ||z||_F, delta_j = eps ||z|| / sqrt 2 on both
 * unfoldings, each rank the smallest r >= 1 whose discarded singular values
 * have sum of squares <= delta^2.  eps <= 0 keeps every nonzero singular
 * value.  norm_before = ||z||, norm_after = ||T(z)|| (either may be NULL). */
int tt_round(tt_ctx* ctx, const tt_t* in, double eps, tt_t** out,
             double* norm_before, double* norm_after);

/* T_eps(in) written into the existing train `out` (same mode sizes), within its
 * rank capacities.  If a rank of T_eps(in) exceeds out's capacity, out holds the
 * truncation to the capacity (the leading singular triplets of each unfolding;
 * the eps bound then does not hold) and the call returns TT_ERANK.  `in` and
 * `out` may not be the same train. */
int tt_round_to(tt_ctx* ctx, const tt_t* in, double eps, tt_t* out, double* norm_before,
                double* norm_after);

/* Randomized T_eps (an opt-in variant of Section 4.1's truncation): when the second
 * rank exceeds 256, a Gaussian sketch (Khatri-Rao test matrix over time and gPC modes,
 * counter-based draws from `seed`) of the second unfolding's row space replaces the
 * last core by an orthonormal basis of ell columns, ell = max(128, R2 / 4) doubling
 * until 8 Gaussian probes estimate the energy the basis misses below 0.1% of
 * eps^2 ||z||^2; the deterministic T_eps then truncates the small train with the budget
 * that is left.  The bound ||T(z) - z|| <= eps ||z|| then holds with high probability;
 * ranks can differ from tt_round's by the rank-decision noise.  Smaller ranks, or a
 * sketch that would not be narrower than R2, take tt_round.  sketch (may be NULL):
 * the width used (R2 when deterministic). */
int tt_round_randomized(tt_ctx* ctx, const tt_t* in, double eps, unsigned long long seed, tt_t** out,
                        double* norm_before, double* norm_after, int* sketch);

/* <vec a, vec b> (Section 4.1) into *out (host). */
int tt_dot(tt_ctx* ctx, const tt_t* a, const tt_t* b, double* out);

/* ||vec a||_F into *out (host): the square root of <a, a> by the same core
 * contractions as tt_dot. */
int tt_norm(tt_ctx* ctx, const tt_t* a, double* out);

/* alpha a + beta b by concatenating cores (ranks add, Section 4.1); eps > 0 then
 * truncates the sum with T_eps, eps <= 0 returns it untruncated. */
int tt_axpby(tt_ctx* ctx, double alpha, const tt_t* a, double beta, const tt_t* b, double eps,
             tt_t** out);

/* <vec a, vec b> into *out (host), like tt_dot, for callers that cannot allocate
 * device memory at the call: a process that has given its whole device memory to
 * its own pool up front (any further cudaMalloc fails), or a latency-critical loop
 * that must not enter an allocator.  The paper has no counterpart of this entry
 * point.  All scratch lives in one static device array of 2^21 doubles (16 MiB per
 * device, held for the life of the process); nothing is allocated.  Ranks whose
 * intermediates need more than that, r1a*r1b + r1a*n_xi*r2b + 2*r2a*r2b + 1
 * doubles, are rejected with TT_EINVAL and a message naming the sizes.  The
 * scratch is shared by every caller on a device: calls that overlap in time
 * (other threads, streams or contexts on the same device) race on it and return
 * wrong values, so serialise them.  Synchronises the context stream. */
int tt_dot_noalloc(tt_ctx* ctx, const tt_t* a, const tt_t* b, double* out);

/* ---- the discrete problem (Sections 3, 5.1) -------------------------------- */

/* Statement of the discrete all-at-once problem.  All arrays are host memory
 * and are copied.  Node numbering and element orders follow the mesh
 * generator: a Q2 element lists nodes a + 3b (a along x1, b along x2,
 * a,b in {0,1,2}); its Q1 vertices a + 2b (a,b in {0,1}); elements are
 * squares of side h.  nu holds nodal viscosity fields on the Q1 vertices:
 * nu[0] the mean nu0, nu[l] = nu0 sigma sqrt(beta_l) a_l (l = 1..m); they are
 * bilinear on each element.  multi_index lists the gPC multi-indices
 * (n_xi x m, row-major); index 0 must be the constant polynomial.
 * tprofile[k] is the inflow time factor at t_{k+1}; inflow[j] is the steady
 * x1-velocity at Dirichlet node j (0 on walls). */
typedef struct {
    int n_nodes, n_elem, n_pnodes;
    double h;
    const double* xy;               /* n_nodes x 2 */
    const long long* elem_q2;       /* n_elem x 9 */
    const long long* elem_q1;       /* n_elem x 4 */
    const unsigned char* dirichlet; /* n_nodes, 1 = Dirichlet */
    const double* inflow;           /* n_nodes */
    int m, n_xi;
    const long long* multi_index;   /* n_xi x m */
    const double* nu;               /* (m + 1) x n_pnodes */
    int n_t;
    double tau;
    const double* tprofile;         /* n_t */
} tt_problem_desc;

/* Build the device-resident discretisation: Q2-Q1 matrices of eq. (mat_entries)
 * and B (free and Dirichlet column blocks), the gPC matrices G_l, H_l
 * (Section 3.2), the lifting of the Dirichlet data and the right-hand side. */
int tt_problem_create(tt_ctx* ctx, const tt_problem_desc* desc, tt_problem** out);
int tt_problem_destroy(tt_problem* prob);
/* n_u = 2 n_v free velocity dofs, n_p pressure dofs, n_xi, n_t. */
int tt_problem_sizes(const tt_problem* prob, int* n_u, int* n_p, int* n_v, int* n_xi,
                     int* n_t, int* n_nodes);
/* Copy out an assembled scalar matrix in CSR form over free dofs (rows) and
 * free (block 0) or Dirichlet (block 1) columns, for verification.  which:
 * 0 = M, 1 + l = A_l, 100 = B_x1, 101 = B_x2 (pressure rows), 200 = M_p, 201 =
 * A_p,0 (Q1 pressure space, block 0 only).  Pass NULL buffers to query nnz / rows
 * first. */
int tt_problem_matrix(tt_ctx* ctx, const tt_problem* prob, int which, int block,
                      int* n_rows, int* n_cols, int* nnz, int* rowptr, int* colidx,
                      double* vals);

/* Right-hand side f = (f^u, f^p) of the all-at-once system (Dirichlet data). */
int tt_rhs(tt_ctx* ctx, tt_problem* prob, tt_t** fu, tt_t** fp);
/* Full-node velocity w = E u + u_D (n_x = 2 n_nodes, ranks + 1). */
int tt_full_velocity(tt_ctx* ctx, tt_problem* prob, const tt_t* u, tt_t** w);

/* ---- operators (eq. F, eq. N_kron, Section 5.2) ------------------------------ */

enum { TT_OP_FULL = 0, TT_OP_MEAN = 1 };

/* Operator of the linear system at a Picard step: FULL is
 * [[F(w) + C, B^T], [B, 0]]; MEAN is the velocity block F_0 + C of Section 5.2.
 * w: full-node convection train (tt_full_velocity, usually truncated), or NULL
 * for the Stokes problem (N = 0).  The operator keeps a copy of what it needs,
 * including the preconditioner factors of Section 5 (built on first use). */
int tt_op_create(tt_ctx* ctx, tt_problem* prob, const tt_t* w, int which, tt_op** out);
int tt_op_destroy(tt_op* op);

/* (out_u, out_p) = L [u; p] for a FULL operator (p may not be NULL), or
 * out_u = (F_0 + C) u for a MEAN operator (p, out_p ignored).  eps > 0 rounds
 * each output train with T_eps. */
int tt_matvec(tt_ctx* ctx, const tt_op* op, const tt_t* u, const tt_t* p, double eps,
              tt_t** out_u, tt_t** out_p);

/* ---- preconditioners (eq. prec, Section 5) ---------------------------------- */

enum {
    TT_PREC_LSC = 0,      /* mean-based LSC Schur approximation, eq. (mean_lsc), with the
                             (1,1) block solved by inner low-rank GMRES on eq. (11_sys)
                             preconditioned by eq. (11_prec) */
    TT_PREC_LEARNED = 1,  /* the same, with the spatial factor K^-1 of eq. (11_prec)
                             replaced by a trained network (tt_net); an inner solve that
                             misses tol_inner with it within max(4, maxit_inner / 5)
                             iterations is redone with the exact K^-1 */
    TT_PREC_PCD = 2       /* mean-based PCD Schur approximation, eq. (mean_pcd):
                             -(B M_*^-1 B^T)^-1 (F_p,0 + C_p) M_p*^-1 with the Q1
                             pressure-space mass, mean diffusion and mean convection
                             (natural boundary conditions), M_p* = diag(M_p); the (1,1)
                             block as for TT_PREC_LSC */
};

typedef struct {
    double eps;           /* truncation inside the preconditioner (the LSC product, the
                             inner GMRES) */
    double tol_inner;     /* inner solve stopping ||y - (F_0 + C) v|| <= tol_inner ||y|| */
    int maxit_inner;      /* inner GMRES iteration cap (<= 63) */
    const tt_net* net;    /* TT_PREC_LEARNED: the network (kept by reference; it must
                             outlive the preconditioner); NULL otherwise */
} tt_prec_opts;

/* Preconditioner of the given kind for a FULL operator (its convection field). */
int tt_prec_create(tt_ctx* ctx, tt_op* op, int kind, const tt_prec_opts* opts, tt_prec** out);
int tt_prec_destroy(tt_prec* prec);

/* Block triangular preconditioner of eq. (prec): p = -S^-1 a_p,
 * u = (F_0 + C)^-1 (a_u - B^T p), applied to (a_u, a_p).  inner_its: iterations of
 * the inner solve(s); fallbacks: learned inner solves redone with the exact K^-1
 * (either pointer may be NULL). */
int tt_prec_apply(tt_ctx* ctx, tt_prec* prec, const tt_t* au, const tt_t* ap, tt_t** u, tt_t** p,
                  int* inner_its, int* fallbacks);

/* ---- learned mean-Oseen solve (no counterpart in the paper) ------------------ */

/* A convolutional network Phi that approximates K^-1 r for the spatial factor
 * K = tau^-1 M + A_0 + N(w_avg) of eq. (11_prec), on the lattice of the problem's
 * velocity nodes (spacing h/2 over the bounding box).  Layers: `depth` 3x3
 * convolutions with zero padding, channels 5 -> C -> ... -> C -> 2, ReLU after all
 * but the last.  Input channels: the two residual components divided by the
 * residual's norm s, the two components of w_avg, the domain mask; output: the two
 * correction components at the free nodes, multiplied by s.  Weights are kept in
 * FP32 and used in BF16; products accumulate in FP32.
 * params (host, FP32): per layer l its weights W_l[out][in][3][3] then its biases
 * b_l[out], layers in order (tt_net_info gives the count).  The network belongs to
 * the problem's mesh; its buffers come from ctx, which must outlive it. */
int tt_net_create(tt_ctx* ctx, const tt_problem* prob, int channels, int depth, const float* params,
                  tt_net** out);
int tt_net_destroy(tt_net* net);
int tt_net_info(const tt_net* net, int* nparams, int* nx, int* ny);
/* on != 0 (the default): convolutions with a multiple of 16 (<= 256) output
 * channels run on the tensor cores as implicit GEMMs with BF16 activations and
 * weights and FP32 accumulation; 0: every convolution on CUDA cores with FP32
 * activations (BF16 weights, FP32 accumulation). */
int tt_net_set_tensor_cores(tt_net* net, int on);
/* Current FP32 parameters (layout as in tt_net_create) into params (host). */
int tt_net_get_params(tt_ctx* ctx, const tt_net* net, float* params);

/* Residual blocks R (and targets T) are n_u x count, row-major (element (i, b) at
 * i * count + b, rows in the velocity order of the trains), host memory
 * (on_device = 0) or device memory (1).  w_avg comes from the operator's
 * convection field (zero for a Stokes operator). */

/* out = Phi(r_b) for every column b (same layout as R). */
int tt_net_apply(tt_ctx* ctx, const tt_net* net, const tt_op* op, const double* R, int count, int on_device,
                 double* out);
/* Training loss (1/count) sum_b ||Phi(r_b) - t_b||^2 / ||t_b||^2 and its gradient with
 * respect to the parameters (host FP32, layout of tt_net_create; may be NULL),
 * without changing the network. */
int tt_net_loss_grad(tt_ctx* ctx, tt_net* net, const tt_op* op, const double* R, const double* T, int count,
                     int on_device, double* loss, float* grads);

typedef struct {
    int epochs;          /* passes over the pairs */
    int batch;           /* pairs per Adam step (a trailing partial batch is skipped) */
    float lr;            /* Adam step size (beta1 0.9, beta2 0.999, eps 1e-8) */
    int smooth_max;      /* residual group g of smooth_max + 1 equal contiguous groups gets g
                            weighted-Jacobi sweeps r <- r - omega D^-1 K r before its target */
    float omega;
} tt_train_opts;

/* Train the network on the pairs (r_b, K^-1 r_b): the residuals R are first
 * smoothed (tt_train_opts), the targets come from the exact banded solve with the
 * operator's K (FP64); then `epochs` passes of Adam steps over consecutive batches
 * in the given order.  epoch_loss (host, `epochs` values, may be NULL): mean batch
 * loss of every pass. */
int tt_net_train(tt_ctx* ctx, tt_net* net, tt_op* op, const double* R, int count, int on_device,
                 const tt_train_opts* opts, double* epoch_loss);

/* Nonlinear residual r = f - A(w)[u; p], w = E u + u_D untruncated
 * (Section 4.3), truncated with eps; *norm = ||T(r)||. */
int tt_residual(tt_ctx* ctx, tt_problem* prob, const tt_t* u, const tt_t* p, double eps,
                tt_t** ru, tt_t** rp, double* norm);

/* ---- solvers (Algorithms 4.2, 3.1) ----------------------------------------- */

enum { TT_FP64 = 0, TT_MIXED = 1 };
enum { TT_ROUND_EXACT = 0, TT_ROUND_RANDOMIZED = 1 };

typedef struct {
    double tol_picard;   /* Picard stopping ||r|| <= tol_picard ||f|| */
    double tol_gmres;    /* outer GMRES stopping, relative to ||b|| */
    double eps_gmres;    /* truncation in GMRES (and the inner solve) */
    double eps_soln;     /* truncation of the Picard iterates, eq. (eps_soln) */
    double eps_conv;     /* truncation of the convection field, eq. (eps_conv) */
    double tol_inner;    /* inner (F_0 + C) solve stopping, Section 5.3 */
    int maxit_picard, maxit_gmres, maxit_inner;
    int precision;       /* TT_FP64: FP64 throughout; TT_MIXED: inside GMRES (matvecs,
                            truncations, the preconditioner) SpMM, GEMM, Householder R
                            factors and banded solves compute in FP32 on FP64-stored
                            trains, while inner products, Hessenberg least squares, the
                            SVDs of the truncations, band factorisations, the Picard
                            residual and the Picard-level truncations stay FP64 */
    const tt_net* learned;  /* non-NULL: TT_PREC_LEARNED preconditioner with this network
                               at every Picard step (exact fallback); NULL: TT_PREC_LSC */
    const tt_t* init_u;     /* non-NULL (with init_p): start Algorithm 3.1 from this
                               iterate instead of the Stokes solve (resume a solve) */
    const tt_t* init_p;
    int rounding;           /* TT_ROUND_EXACT: every truncation by T_eps; TT_ROUND_RANDOMIZED:
                               the truncations inside GMRES (and the preconditioner) by
                               tt_round_randomized, the Picard-level ones exact */
    int schur;              /* Schur complement approximation of the preconditioner built
                               from these options: TT_PREC_LSC (eq. mean_lsc, 0) or
                               TT_PREC_PCD (eq. mean_pcd); other values: TT_EINVAL */
} tt_solver_opts;

typedef struct {
    int its;             /* iterations taken */
    double res0;         /* ||s_0|| */
    double res;          /* ||s_k|| at exit */
    int inner_its;       /* total inner iterations of the preconditioner */
    int fallbacks;       /* learned inner solves redone with the exact K^-1 */
} tt_gmres_stats;

#define TT_MAX_PICARD 64
typedef struct {
    int picard_its;
    int stokes_its;
    double fnorm;
    double res[TT_MAX_PICARD + 1];        /* ||r^(i)||, i = 0..picard_its */
    int gmres_its[TT_MAX_PICARD + 1];     /* per Picard step (index 0: Stokes) */
    int inner_its[TT_MAX_PICARD + 1];
    int ranks[TT_MAX_PICARD + 1][4];      /* u (k1,k2), p (k1,k2) after each step */
    int conv_ranks[TT_MAX_PICARD + 1][2]; /* truncated convection field */
    int fallbacks[TT_MAX_PICARD + 1];     /* learned inner solves redone exactly */
} tt_picard_stats;

/* Low-rank flexible GMRES (Algorithm 4.2) for op [z_u; z_p] = [b_u; b_p] with
 * the preconditioner prec (NULL: TT_PREC_LSC built from opts), z_0 = 0, stop
 * when ||s_k|| <= tol_gmres * bnorm (bnorm <= 0: use ||b||).  Returns
 * TT_ENOCONV (with the last iterate) if maxit_gmres is reached first. */
int tt_gmres(tt_ctx* ctx, tt_op* op, tt_prec* prec, const tt_solver_opts* opts, const tt_t* bu,
             const tt_t* bp, double bnorm, tt_t** zu, tt_t** zp, tt_gmres_stats* stats);

/* Truncated inexact Picard iteration (Algorithm 3.1, eq. eps_soln, eq. eps_conv,
 * Section 5.2): Stokes initial iterate (or opts->init_u, init_p), then correction
 * solves until ||r|| <= tol_picard ||f||.  Returns the velocity and pressure
 * trains; stats index 0 is the Stokes solve (zero when resumed). */
int picard_solve(tt_ctx* ctx, tt_problem* prob, const tt_solver_opts* opts, tt_t** u,
                 tt_t** p, tt_picard_stats* stats);

/* Batched form: nprob independent problems solved concurrently, each exactly as
 * picard_solve (Algorithm 3.1) with its own options opts[i].  The paper has no
 * batched form.  Every problem must belong to a different context (its own
 * stream); each solve runs on its own host thread, so the latency-bound launches
 * of one solve overlap those of the others on the GPU.  Outputs per problem:
 * u[i], p[i] (NULL when status[i] is an error other than TT_ENOCONV), stats[i],
 * status[i] (as picard_solve returns it) and, if seconds is not NULL,
 * seconds[i] = wall time of that solve.  Returns TT_OK when every status is
 * TT_OK, TT_EINVAL for bad arguments (shared contexts included, nothing run),
 * else the first failing status. */
int picard_solve_batched(int nprob, tt_problem* const* probs, const tt_solver_opts* opts,
                         tt_t** u, tt_t** p, tt_picard_stats* stats, int* status,
                         double* seconds);

#ifdef __cplusplus
}
#endif
#endif /* TT_STOCHNS_H */
