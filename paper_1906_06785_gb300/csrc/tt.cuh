// Tensor-train operations of Section 4.1 on device-resident trains.
#pragma once
#include "la.cuh"

namespace tt {

// One summand of a concatenation: coef * (dcoef ? *dcoef : 1) * t.
struct Summand {
    double coef;
    const double* dcoef;   // device scalar or nullptr
    const tt_t* t;
};

// sum_i coef_i t_i by concatenating cores (ranks add).
TTPtr concat(tt_ctx* c, const std::vector<Summand>& terms);

// Truncations with eps at or above this use the Gram route (see tt.cu).
constexpr double kGramMinEps = 5e-6;

// T_eps(z); fills the norms before / after truncation.
struct RoundOut {
    double nrm_before = 0.0, nrm_after = 0.0;
    int capped = 0;   // nonzero: a rank was cut to its cap (the error bound may not hold)
};
// cap1, cap2 > 0 bound the output ranks (the truncation then keeps the leading
// singular triplets up to the cap and reports it in info->capped).
TTPtr round_tt(tt_ctx* c, const tt_t* z, double eps, RoundOut* info = nullptr, int cap1 = 0, int cap2 = 0);

// T_eps by round_rand when the context's randomized flag is set, else round_tt.
TTPtr round_any(tt_ctx* c, const tt_t* z, double eps, RoundOut* info = nullptr);

// T_eps of a velocity train u and a pressure train p, the two truncations running
// concurrently (the pressure one on the context's side stream).
void round_pair(tt_ctx* c, const tt_t* u, const tt_t* p, double eps, TTPtr* ru, TTPtr* rp, RoundOut* iu,
                RoundOut* ip);

// Randomized T_eps (rround.cu): trains whose second rank exceeds kRandMinRank are first
// compressed by a Gaussian sketch of ell columns (ell doubling until probes estimate the
// missed energy below 0.1% of eps^2 ||z||^2), then truncated deterministically; smaller
// trains, and sketches that would not be narrower than R2, take round_tt.  seed selects
// the draws; ell_used (may be null) reports the sketch width (R2: deterministic).
constexpr int kRandMinRank = 256;
TTPtr round_rand(tt_ctx* c, const tt_t* z, double eps, uint64_t seed, RoundOut* info = nullptr,
                 int* ell_used = nullptr);

// <vec a, vec b> written to the device scalar *dout.
void dot_dev(tt_ctx* c, const tt_t* a, const tt_t* b, double* dout);
double dot_host(tt_ctx* c, const tt_t* a, const tt_t* b);

// Copy the cores of s into t (t's capacities must hold s's ranks; t takes s's ranks).
void copy_cores(tt_ctx* c, const tt_t* s, tt_t* t);

// Copy of a train (same ranks), optionally scaled by a host scalar.
TTPtr clone(tt_ctx* c, const tt_t* t, double scale = 1.0);

// Rank-1 zero train.
TTPtr zeros(tt_ctx* c, int n_t, int n_xi, int n_x);

}  // namespace tt
