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
constexpr int kSingleCtasPerSm = 1;    // resident CTAs per SM the single-period variant is built for

// One instance as the solver kernel sees it (device memory).  All per-asset
// arrays have row stride np (n rounded up to a multiple of 32).  Panels are
// stored as S (double, float or bfloat16) and multiplied in M (double or
// float); the iterate state and every elementwise update are FP64.
template <class M, class S>
struct Inst {
    int n, k, m, P, R, multi, np, omega_diag;
    const S* Ft;          // k x np factor-major F^T, followed by np x k asset-major F
    const S* At;          // m x np exposure rows, followed by np x m asset-major A^T
    const double* Om;     // k x k, or k diagonal entries
    const double* alpha;  // P x np
    const double* Dp;     // P x np
    const double* Dmax;   // np       max over periods of D (for the Lipschitz bound)
    const double* c1;     // R x np   lambda2 * s
    const double* c2;     // R x np   lambda3 * q
    const double* w0;     // np
    const double* cen;    // np       risk centre: w_T (multi) or 0 (single)
    const double* alphaT; // np       alpha at t = T (multi) or unused
    const double* L;      // m
    const double* U;      // m
    double kappa, d;
    double GMV;
    // iterate storage (workspace)
    double *x, *x0, *xb, *xn, *v;      // P x np
    double *yD, *yD0, *yDb, *yDn;      // R x np
    double* yA0;                       // P x m anchor of the replicated y_A
    double *pv1, *pv2;                 // np power-iteration vectors
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
    double beta;
    int power_iters;
    int* queue;          // device counter of the next instance (zero at launch); teams take
                         // instances from it in table order
};

// Shared-memory bytes the solver kernel needs for these sizes.
size_t solver_smem_bytes(int P, int k, int m, int omega_diag, size_t matvec_size);

// Launch the team kernel over `count` instances (insts is a device array).
// G = CTAs per instance (cluster size), nteams = concurrent teams; single =
// every instance is single-period (the variant built for P = 1).
template <class M, class S>
cudaError_t launch_solver(const Inst<M, S>* insts, int count, const Params& prm, int G, int nteams,
                          size_t smem, bool single, cudaStream_t stream);

template <class M, class S>
cudaError_t max_teams(int G, size_t smem, bool single, int* out);

}  // namespace ff
