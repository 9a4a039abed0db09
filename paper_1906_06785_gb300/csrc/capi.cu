// extern "C" entry points declared in include/tt_stochns.h.  Every entry point
// catches the library's exceptions and turns them into status codes.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "solver.cuh"

using namespace tt;

namespace tt {
void check_status(tt_ctx* c) {
    int s = DEV_OK;
    read_back(c, c->dstatus, &s, 1);
    if (s != DEV_OK) {
        CUDA_CHECK(cudaMemsetAsync(c->dstatus, 0, sizeof(int), c->stream));
        if (s == DEV_TIMEOUT) TT_THROW(TT_ETIMEOUT, "a device-side wait ran out of its budget");
        TT_THROW(TT_ENAN, "zero or non-finite pivot / value met on the device");
    }
}
int max_cluster_ctas(tt_ctx* c, const void* kernel, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(c->device, kernel, threads, smem);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int best = 0;
    for (int size : {16, 8}) {
        if (size > 8 && cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(size);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = size;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) == cudaSuccess && n > 0) {
            best = size;
            break;
        }
        (void)cudaGetLastError();
    }
    cache[key] = best;
    return best;
}

tt_ctx* side_ctx(tt_ctx* c) {
    if (c->side) return c->side;
    tt_ctx* s = new tt_ctx;
    try {
        s->device = c->device;
        s->nsm = c->nsm;
        s->alloc_fn = c->alloc_fn;
        s->free_fn = c->free_fn;
        s->alloc_user = c->alloc_user;
        s->gram_ok = c->gram_ok;
        s->wait_limit = c->wait_limit;
        CUDA_CHECK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
        CUDA_CHECK(cudaMallocHost(&s->pinned, 4096));
        CUDA_CHECK(cudaMalloc((void**)&s->dstatus, sizeof(int)));
        CUDA_CHECK(cudaMalloc((void**)&s->dbarrier, 4 * sizeof(unsigned)));
        CUDA_CHECK(cudaMemset(s->dstatus, 0, sizeof(int)));
        CUDA_CHECK(cudaMemset(s->dbarrier, 0, 4 * sizeof(unsigned)));
        CUDA_CHECK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
        CUDA_CHECK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    } catch (...) {
        if (s->stream) cudaStreamDestroy(s->stream);
        if (s->pinned) cudaFreeHost(s->pinned);
        if (s->dstatus) cudaFree(s->dstatus);
        if (s->dbarrier) cudaFree(s->dbarrier);
        delete s;
        throw;
    }
    c->side = s;
    return s;
}

void destroy_side(tt_ctx* c) {
    tt_ctx* s = c->side;
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    cudaStreamDestroy(s->stream);
    cudaFreeHost(s->pinned);
    cudaFree(s->dstatus);
    cudaFree(s->dbarrier);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    delete s;
    c->side = nullptr;
}

static cudaEvent_t ev_get(tt_ctx* c) {
    if (!c->pd.pool.empty()) {
        cudaEvent_t e = c->pd.pool.back();
        c->pd.pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    CUDA_CHECK(cudaEventCreate(&e));
    return e;
}

ProfScope::ProfScope(tt_ctx* ctx, int s, double flops, double bytes) : c(ctx), slot(s) {
    if (!c->prof) return;
    c->pd.flops[s] += flops;
    c->pd.bytes[s] += bytes;
    c->pd.n[s] += 1;
    a = ev_get(c);
    b = ev_get(c);
    cudaEventRecord(a, c->stream);
}
ProfScope::~ProfScope() {
    if (!a) return;
    cudaEventRecord(b, c->stream);
    c->pd.pending[slot].push_back({a, b});
}

void prof_resolve(tt_ctx* c) {
    CUDA_CHECK(cudaStreamSynchronize(c->stream));
    for (int s = 0; s < PROF_NSLOTS; ++s) {
        for (auto& pr : c->pd.pending[s]) {
            float ms = 0.f;
            CUDA_CHECK(cudaEventElapsedTime(&ms, pr.first, pr.second));
            c->pd.ms[s] += ms;
            c->pd.pool.push_back(pr.first);
            c->pd.pool.push_back(pr.second);
        }
        c->pd.pending[s].clear();
    }
}
}  // namespace tt

// A preconditioner object: the kind and options, applied through LSCPrec.
struct tt_prec {
    tt_ctx* c = nullptr;
    tt_op* op = nullptr;
    int kind = TT_PREC_LSC;
    tt_prec_opts o{};
    LSCPrec make() const { return LSCPrec{c, op, o.eps, o.tol_inner, o.maxit_inner, o.net, kind == TT_PREC_PCD}; }
};

#define API_BEGIN(ctx) \
    tt_ctx* _ctx = (ctx); \
    try {
#define API_END                                             \
    return TT_OK;                                           \
    }                                                       \
    catch (const tt::Error& e) {                            \
        if (_ctx) _ctx->err = e.what();                     \
        return e.code;                                      \
    }                                                       \
    catch (const std::exception& e) {                       \
        if (_ctx) _ctx->err = e.what();                     \
        return TT_ECUDA;                                    \
    }

extern "C" {

int tt_ctx_create(void* stream, tt_alloc_fn alloc, tt_free_fn free_fn, void* user, tt_ctx** out) {
    if (!out) return TT_EINVAL;
    *out = nullptr;
    if ((alloc == nullptr) != (free_fn == nullptr)) return TT_EINVAL;
    tt_ctx* c = new tt_ctx;
    try {
        c->stream = (cudaStream_t)stream;
        c->alloc_fn = alloc;
        c->free_fn = free_fn;
        c->alloc_user = user;
        CUDA_CHECK(cudaGetDevice(&c->device));
        CUDA_CHECK(cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device));
        int coop = 0;
        CUDA_CHECK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device));
        if (!coop) TT_THROW(TT_ECUDA, "device does not support cooperative launches");
        CUDA_CHECK(cudaMallocHost(&c->pinned, 4096));
        CUDA_CHECK(cudaMalloc((void**)&c->dstatus, sizeof(int)));
        CUDA_CHECK(cudaMalloc((void**)&c->dbarrier, 4 * sizeof(unsigned)));
        CUDA_CHECK(cudaMemset(c->dstatus, 0, sizeof(int)));
        CUDA_CHECK(cudaMemset(c->dbarrier, 0, 4 * sizeof(unsigned)));
        CUDA_CHECK(cudaMalloc((void**)&c->dprof_flops, PROF_NSLOTS * sizeof(double)));
        CUDA_CHECK(cudaMemset(c->dprof_flops, 0, PROF_NSLOTS * sizeof(double)));
        cudaMemPool_t pool;
        CUDA_CHECK(cudaDeviceGetDefaultMemPool(&pool, c->device));
        unsigned long long thr = ~0ULL;
        CUDA_CHECK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    } catch (const tt::Error& e) {
        if (c->pinned) cudaFreeHost(c->pinned);
        if (c->dstatus) cudaFree(c->dstatus);
        if (c->dbarrier) cudaFree(c->dbarrier);
        delete c;
        return e.code;
    }
    *out = c;
    return TT_OK;
}

int tt_ctx_destroy(tt_ctx* c) {
    if (!c) return TT_EINVAL;
    cudaStreamSynchronize(c->stream);
    destroy_side(c);
    try { prof_resolve(c); } catch (...) {}
    for (auto e : c->pd.pool) cudaEventDestroy(e);
    cudaFreeHost(c->pinned);
    cudaFree(c->dstatus);
    cudaFree(c->dbarrier);
    cudaFree(c->dprof_flops);
    delete c;
    return TT_OK;
}

const char* tt_last_error(const tt_ctx* c) { return c ? c->err.c_str() : "null context"; }

long long tt_ctx_launches(const tt_ctx* c) { return c ? c->launches : -1; }

int tt_ctx_set_wait_limit(tt_ctx* c, long long polls) {
    if (!c || polls < 0) return TT_EINVAL;
    c->wait_limit = polls;
    if (c->side) c->side->wait_limit = polls;
    return TT_OK;
}

int tt_ctx_profile(tt_ctx* ctx, int enable) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx, "null context");
    prof_resolve(ctx);
    for (int s = 0; s < PROF_NSLOTS; ++s) {
        ctx->pd.ms[s] = ctx->pd.flops[s] = ctx->pd.bytes[s] = 0.0;
        ctx->pd.n[s] = 0;
    }
    CUDA_CHECK(cudaMemsetAsync(ctx->dprof_flops, 0, PROF_NSLOTS * sizeof(double), ctx->stream));
    ctx->prof = enable != 0;
    API_END
}

int tt_ctx_prof_read(tt_ctx* ctx, int slot, long long* n, double* ms, double* flops, double* bytes) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && slot >= 0 && slot < PROF_NSLOTS, "bad profiling slot");
    prof_resolve(ctx);
    double dev[PROF_NSLOTS];
    read_back(ctx, ctx->dprof_flops, dev, PROF_NSLOTS);
    if (n) *n = ctx->pd.n[slot];
    if (ms) *ms = ctx->pd.ms[slot];
    if (flops) *flops = ctx->pd.flops[slot] + dev[slot];
    if (bytes) *bytes = ctx->pd.bytes[slot];
    API_END
}

int tt_create(tt_ctx* ctx, int n_t, int n_xi, int n_x, int r1, int r2, int rcap1, int rcap2, int dtype,
              const double* z1, const double* z2, const double* z3, int src_on_device, tt_t** out) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && out && z1 && z2 && z3, "null argument");
    TT_REQUIRE(dtype == TT_F64, "unsupported train dtype %d (TT_F64 only)", dtype);
    *out = nullptr;
    TTPtr t = wrap(tt_alloc(ctx, n_t, n_xi, n_x, r1, r2, rcap1, rcap2));
    const cudaMemcpyKind k = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CUDA_CHECK(cudaMemcpyAsync(t->z1, z1, (size_t)n_t * r1 * sizeof(double), k, ctx->stream));
    CUDA_CHECK(cudaMemcpyAsync(t->z2, z2, (size_t)r1 * n_xi * r2 * sizeof(double), k, ctx->stream));
    CUDA_CHECK(cudaMemcpyAsync(t->z3, z3, (size_t)n_x * r2 * sizeof(double), k, ctx->stream));
    if (!src_on_device) CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    *out = t.release();
    API_END
}

int tt_destroy(tt_t* t) {
    if (!t) return TT_EINVAL;
    tt_free(t);
    return TT_OK;
}

int tt_shape(const tt_t* t, int* n_t, int* n_xi, int* n_x, int* r1, int* r2) {
    if (!t) return TT_EINVAL;
    if (n_t) *n_t = t->n_t;
    if (n_xi) *n_xi = t->n_xi;
    if (n_x) *n_x = t->n_x;
    if (r1) *r1 = t->r1;
    if (r2) *r2 = t->r2;
    return TT_OK;
}

int tt_capacity(const tt_t* t, int* rcap1, int* rcap2) {
    if (!t) return TT_EINVAL;
    if (rcap1) *rcap1 = t->cap1;
    if (rcap2) *rcap2 = t->cap2;
    return TT_OK;
}

int tt_get_cores(tt_ctx* ctx, const tt_t* t, double* z1, double* z2, double* z3, int dst_on_device) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && t, "null argument");
    const cudaMemcpyKind k = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (z1) CUDA_CHECK(cudaMemcpyAsync(z1, t->z1, (size_t)t->n_t * t->r1 * sizeof(double), k, ctx->stream));
    if (z2) CUDA_CHECK(cudaMemcpyAsync(z2, t->z2, (size_t)t->r1 * t->n_xi * t->r2 * sizeof(double), k, ctx->stream));
    if (z3) CUDA_CHECK(cudaMemcpyAsync(z3, t->z3, (size_t)t->n_x * t->r2 * sizeof(double), k, ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    API_END
}

int tt_round(tt_ctx* ctx, const tt_t* in, double eps, tt_t** out, double* nb, double* na) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && in && out, "null argument");
    RoundOut info;
    TTPtr r = round_tt(ctx, in, eps, &info);
    if (nb) *nb = info.nrm_before;
    if (na) *na = info.nrm_after;
    *out = r.release();
    API_END
}

int tt_round_to(tt_ctx* ctx, const tt_t* in, double eps, tt_t* out, double* nb, double* na) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && in && out, "null argument");
    TT_REQUIRE(in != out, "tt_round_to: input and output are the same train");
    TT_REQUIRE(in->n_t == out->n_t && in->n_xi == out->n_xi && in->n_x == out->n_x,
               "tt_round_to: mode sizes differ");
    RoundOut info;
    TTPtr r = round_tt(ctx, in, eps, &info, out->cap1, out->cap2);
    copy_cores(ctx, r.get(), out);
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    if (nb) *nb = info.nrm_before;
    if (na) *na = info.nrm_after;
    if (info.capped) {
        ctx->err = "tt_round_to: a rank of the truncation exceeds the output capacity; output truncated to it";
        return TT_ERANK;
    }
    API_END
}

int tt_round_randomized(tt_ctx* ctx, const tt_t* in, double eps, unsigned long long seed, tt_t** out, double* nb,
                        double* na, int* sketch) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && in && out, "null argument");
    RoundOut info;
    TTPtr r = round_rand(ctx, in, eps, seed, &info, sketch);
    if (nb) *nb = info.nrm_before;
    if (na) *na = info.nrm_after;
    *out = r.release();
    API_END
}

int tt_dot(tt_ctx* ctx, const tt_t* a, const tt_t* b, double* out) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && a && b && out, "null argument");
    *out = dot_host(ctx, a, b);
    API_END
}

int tt_norm(tt_ctx* ctx, const tt_t* a, double* out) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && a && out, "null argument");
    const double d = dot_host(ctx, a, a);
    if (!(d == d) || std::isinf(d)) TT_THROW(TT_ENAN, "non-finite norm");
    *out = std::sqrt(std::max(d, 0.0));
    API_END
}

int tt_axpby(tt_ctx* ctx, double alpha, const tt_t* a, double beta, const tt_t* b, double eps, tt_t** out) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && a && b && out, "null argument");
    TTPtr s = concat(ctx, {Summand{alpha, nullptr, a}, Summand{beta, nullptr, b}});
    if (eps > 0.0) s = round_tt(ctx, s.get(), eps);
    *out = s.release();
    API_END
}

int tt_problem_create(tt_ctx* ctx, const tt_problem_desc* desc, tt_problem** out) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && desc && out, "null argument");
    *out = nullptr;
    std::unique_ptr<tt_problem> P(new tt_problem);
    build_problem(ctx, P.get(), desc);
    make_rhs(ctx, P.get());
    *out = P.release();
    API_END
}

int tt_problem_destroy(tt_problem* p) {
    if (!p) return TT_EINVAL;
    delete p;
    return TT_OK;
}

int tt_problem_sizes(const tt_problem* P, int* n_u, int* n_p, int* n_v, int* n_xi, int* n_t, int* n_nodes) {
    if (!P) return TT_EINVAL;
    if (n_u) *n_u = 2 * P->n_v;
    if (n_p) *n_p = P->n_p;
    if (n_v) *n_v = P->n_v;
    if (n_xi) *n_xi = P->n_xi;
    if (n_t) *n_t = P->n_t;
    if (n_nodes) *n_nodes = P->n_nodes;
    return TT_OK;
}

int tt_problem_matrix(tt_ctx* ctx, const tt_problem* P, int which, int block, int* n_rows, int* n_cols, int* nnz,
                      int* rowptr, int* colidx, double* vals) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && P, "null argument");
    const Csr* pat = nullptr;
    const double* v = nullptr;
    if (which == 100 || which == 101) {
        pat = block == 0 ? &P->BF : &P->BD;
        v = block == 0 ? (which == 100 ? P->Bx_F.p : P->By_F.p) : (which == 100 ? P->Bx_D.p : P->By_D.p);
    } else if (which == 0) {
        pat = block == 0 ? &P->ff : &P->fD;
        v = block == 0 ? P->M_ff.p : P->M_fD.p;
    } else if (which >= 1 && which <= P->m + 1) {
        pat = block == 0 ? &P->ff : &P->fD;
        const size_t nn = std::max(1, pat->nnz);
        v = (block == 0 ? P->A_ff.p : P->A_fD.p) + (which - 1) * nn;
    } else if ((which == 200 || which == 201) && block == 0) {
        pat = &P->pp;
        v = which == 200 ? P->Mp_pp.p : P->Ap_pp.p;
    } else {
        TT_THROW(TT_EINVAL, "unknown matrix id %d", which);
    }
    if (n_rows) *n_rows = pat->n_rows;
    if (n_cols) *n_cols = pat->n_cols;
    if (nnz) *nnz = pat->nnz;
    if (rowptr) CUDA_CHECK(cudaMemcpyAsync(rowptr, pat->rowptr.p, (pat->n_rows + 1) * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    if (colidx && pat->nnz) CUDA_CHECK(cudaMemcpyAsync(colidx, pat->col.p, pat->nnz * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    if (vals && pat->nnz) CUDA_CHECK(cudaMemcpyAsync(vals, v, pat->nnz * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    API_END
}

int tt_rhs(tt_ctx* ctx, tt_problem* P, tt_t** fu, tt_t** fp) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && P && fu && fp, "null argument");
    *fu = clone(ctx, P->fu).release();
    *fp = clone(ctx, P->fp).release();
    API_END
}

int tt_full_velocity(tt_ctx* ctx, tt_problem* P, const tt_t* u, tt_t** w) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && P && u && w, "null argument");
    TT_REQUIRE(u->n_x == 2 * P->n_v, "u must live on the free velocity dofs");
    *w = full_velocity(ctx, P, u).release();
    API_END
}

int tt_op_create(tt_ctx* ctx, tt_problem* P, const tt_t* w, int which, tt_op** out) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && P && out, "null argument");
    TT_REQUIRE(which == TT_OP_FULL || which == TT_OP_MEAN, "unknown operator kind");
    std::unique_ptr<tt_op> op(new tt_op);
    op_init(ctx, op.get(), P, w, which);
    *out = op.release();
    API_END
}

int tt_op_destroy(tt_op* op) {
    if (!op) return TT_EINVAL;
    delete op;
    return TT_OK;
}

int tt_matvec(tt_ctx* ctx, const tt_op* op, const tt_t* u, const tt_t* p, double eps, tt_t** ou, tt_t** op_) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && op && u && ou, "null argument");
    TTPtr a{nullptr, tt_free}, b{nullptr, tt_free};
    if (op->which == TT_OP_FULL) {
        TT_REQUIRE(p && op_, "FULL operator needs p and out_p");
        op_apply(ctx, op, u, p, &a, &b);
    } else {
        op_apply_mean(ctx, op, u, &a);
    }
    if (eps > 0) {
        a = round_tt(ctx, a.get(), eps);
        if (b) b = round_tt(ctx, b.get(), eps);
    }
    *ou = a.release();
    if (op_) *op_ = b.release();
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    API_END
}

int tt_prec_create(tt_ctx* ctx, tt_op* op, int kind, const tt_prec_opts* o, tt_prec** out) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && op && o && out, "null argument");
    *out = nullptr;
    TT_REQUIRE(op->which == TT_OP_FULL, "a preconditioner needs a FULL operator");
    TT_REQUIRE(o->maxit_inner >= 1 && o->maxit_inner <= 63, "maxit_inner must be in [1, 63]");
    TT_REQUIRE(kind == TT_PREC_LSC || kind == TT_PREC_LEARNED || kind == TT_PREC_PCD,
               "unknown preconditioner kind %d", kind);
    TT_REQUIRE(kind != TT_PREC_LEARNED || o->net, "TT_PREC_LEARNED needs a network");
    tt_prec* pr = new tt_prec;
    pr->c = ctx;
    pr->op = op;
    pr->kind = kind;
    pr->o = *o;
    if (kind != TT_PREC_LEARNED) pr->o.net = nullptr;
    *out = pr;
    API_END
}

int tt_prec_destroy(tt_prec* prec) {
    if (!prec) return TT_EINVAL;
    delete prec;
    return TT_OK;
}

int tt_prec_apply(tt_ctx* ctx, tt_prec* prec, const tt_t* au, const tt_t* ap, tt_t** u, tt_t** p, int* inner_its,
                  int* fallbacks) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && prec && au && ap && u && p, "null argument");
    LSCPrec pre = prec->make();
    Vec v;
    v.u = clone(ctx, au);
    v.p = clone(ctx, ap);
    Vec r = pre.apply(v);
    if (inner_its) *inner_its = pre.inner_its;
    if (fallbacks) *fallbacks = pre.fallbacks;
    *u = r.u.release();
    *p = r.p.release();
    CUDA_CHECK(cudaStreamSynchronize(ctx->stream));
    API_END
}

int tt_residual(tt_ctx* ctx, tt_problem* P, const tt_t* u, const tt_t* p, double eps, tt_t** ru, tt_t** rp,
                double* norm) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && P && u && p && ru && rp, "null argument");
    TTPtr a{nullptr, tt_free}, b{nullptr, tt_free};
    const double n = residual(ctx, P, u, p, eps, &a, &b);
    if (norm) *norm = n;
    *ru = a.release();
    *rp = b.release();
    API_END
}

int tt_gmres(tt_ctx* ctx, tt_op* op, tt_prec* prec, const tt_solver_opts* o, const tt_t* bu, const tt_t* bp,
             double bnorm, tt_t** zu, tt_t** zp, tt_gmres_stats* stats) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && op && o && bu && bp && zu && zp, "null argument");
    TT_REQUIRE(op->which == TT_OP_FULL, "tt_gmres needs a FULL operator");
    TT_REQUIRE(o->precision == TT_FP64 || o->precision == TT_MIXED, "unknown precision %d", o->precision);
    TT_REQUIRE(!prec || prec->op == op, "the preconditioner belongs to another operator");
    TT_REQUIRE(o->schur == TT_PREC_LSC || o->schur == TT_PREC_PCD, "schur must be TT_PREC_LSC or TT_PREC_PCD");
    LSCPrec pre = prec ? prec->make()
                       : LSCPrec{ctx, op, o->eps_gmres, o->tol_inner, o->maxit_inner, o->learned,
                                 o->schur == TT_PREC_PCD};
    Vec b;
    b.u = clone(ctx, bu);
    b.p = clone(ctx, bp);
    GmresOut go;
    tt_ctx* c = ctx;
    TT_REQUIRE(o->rounding == TT_ROUND_EXACT || o->rounding == TT_ROUND_RANDOMIZED, "unknown rounding %d",
               o->rounding);
    PrecScope ps(ctx, o->precision == TT_MIXED ? 1 : 0);
    RandScope rs(ctx, o->rounding == TT_ROUND_RANDOMIZED);
    Vec z = gmres(
        ctx, [c, op](const Vec& x) { Vec y; op_apply(c, op, x.u.get(), x.p.get(), &y.u, &y.p); return y; },
        [&pre](const Vec& v) { return pre.apply(v); }, b, o->tol_gmres, o->eps_gmres, o->maxit_gmres, bnorm, &go);
    if (stats) {
        stats->its = go.its;
        stats->res0 = go.res0;
        stats->res = go.res;
        stats->inner_its = pre.inner_its;
        stats->fallbacks = pre.fallbacks;
    }
    *zu = z.u.release();
    *zp = z.p.release();
    if (!go.converged) {
        ctx->err = "GMRES reached maxit";
        return TT_ENOCONV;
    }
    API_END
}

int picard_solve(tt_ctx* ctx, tt_problem* P, const tt_solver_opts* o, tt_t** u, tt_t** p, tt_picard_stats* st) {
    API_BEGIN(ctx)
    TT_REQUIRE(ctx && P && o && u && p && st, "null argument");
    TTPtr a{nullptr, tt_free}, b{nullptr, tt_free};
    picard(ctx, P, o, &a, &b, st);
    *u = a.release();
    *p = b.release();
    if (st->res[st->picard_its] > o->tol_picard * P->fnorm) {
        ctx->err = "Picard reached maxit";
        return TT_ENOCONV;
    }
    API_END
}

int picard_solve_batched(int nprob, tt_problem* const* probs, const tt_solver_opts* opts, tt_t** u, tt_t** p,
                         tt_picard_stats* stats, int* status, double* seconds) {
    if (nprob <= 0 || !probs || !opts || !u || !p || !stats || !status) return TT_EINVAL;
    for (int i = 0; i < nprob; ++i) {
        if (!probs[i] || !probs[i]->ctx) return TT_EINVAL;
        u[i] = nullptr;
        p[i] = nullptr;
        status[i] = TT_OK;
        if (seconds) seconds[i] = 0.0;
    }
    for (int i = 0; i < nprob; ++i)
        for (int j = i + 1; j < nprob; ++j)
            if (probs[i]->ctx == probs[j]->ctx) {
                probs[i]->ctx->err = "picard_solve_batched: two problems share a context (stream)";
                return TT_EINVAL;
            }
    std::vector<std::thread> workers;
    workers.reserve(nprob);
    for (int i = 0; i < nprob; ++i) {
        workers.emplace_back([=]() {
            tt_ctx* c = probs[i]->ctx;
            const auto t0 = std::chrono::steady_clock::now();
            if (cudaSetDevice(c->device) != cudaSuccess) {
                c->err = "picard_solve_batched: cannot make the context's device current";
                status[i] = TT_ECUDA;
                return;
            }
            status[i] = picard_solve(c, probs[i], &opts[i], &u[i], &p[i], &stats[i]);
            cudaStreamSynchronize(c->stream);
            if (seconds) seconds[i] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        });
    }
    for (auto& w : workers) w.join();
    for (int i = 0; i < nprob; ++i)
        if (status[i] != TT_OK) return status[i];
    return TT_OK;
}

}  // extern "C"
