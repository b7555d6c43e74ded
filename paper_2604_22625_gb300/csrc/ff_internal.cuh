// Internal declarations shared by the solver kernels and the C ABI layer.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/flashfolio.h"

namespace ff {

constexpr int kThreads = 256;          // threads per CTA
constexpr int kWarps = kThreads / 32;
constexpr int kPC = 8;                 // periods processed together in a matvec pass
constexpr int kCand = 8;               // threshold candidates per period and search round
constexpr int kMaxRounds = 16;         // threshold search rounds per projection
constexpr int kMaxCluster = 16;

// One instance as the solver kernel sees it (device memory).  All per-asset
// arrays have row stride np (n rounded up to a multiple of 32).
template <class real, class S>
struct Inst {
    int n, k, m, P, R, multi, np, omega_diag;
    const S* Ft;        // k x np   factor loadings, factor-major (F^T)
    const S* At;        // m x np   exposure rows
    const real* Om;     // k x k, or k diagonal entries
    const real* alpha;  // P x np
    const real* Dp;     // P x np
    const real* Dmax;   // np       max over periods of D (for the Lipschitz bound)
    const real* c1;     // R x np   lambda2 * s
    const real* c2;     // R x np   lambda3 * q
    const real* w0;     // np
    const real* cen;    // np       risk centre: w_T (multi) or 0 (single)
    const real* alphaT; // np       alpha at t = T (multi) or nullptr
    const real* L;      // m
    const real* U;      // m
    real kappa, d;
    double GMV;
    // iterate storage (workspace)
    real *x, *x0, *xb, *xn, *v;        // P x np
    real *yD, *yD0, *yDb, *yDn;        // R x np
    real *yA0, *u0, *ax0;              // P x m, P x k, P x m (anchors of the replicated vectors)
    real *pv1, *pv2;                   // np power-iteration vectors
    // outputs
    void* w_out;        // P x n   (out dtype)
    void* yA_out;       // P x m   or nullptr
    void* yD_out;       // R x n   or nullptr
    int out_f64;
    ff_result* res;
};

struct Params {
    double tol;
    long long max_iter;
    double time_limit_ns;
    int check_every;
    double rho;
    double beta_suff, beta_nec;
    double step_fraction;
    int power_iters;
};

// Shared-memory bytes the solver kernel needs for these sizes.
size_t solver_smem_bytes(int P, int k, int m, int omega_diag, size_t real_size);

// Launch the team kernel over `count` instances (insts is a device array).
// G = CTAs per instance (cluster size), nteams = concurrent teams.
template <class real, class S>
cudaError_t launch_solver(const Inst<real, S>* insts, int count, const Params& prm, int G, int nteams,
                          size_t smem, cudaStream_t stream);

template <class real, class S>
cudaError_t max_teams(int G, size_t smem, int* out);

}  // namespace ff
