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

constexpr int kStages = 3;             // bulk-copy ring stages per CTA
constexpr int kMaxTileBytes = 48 * 1024;
constexpr int kSmemLimit = 227 * 1024 - 4096;   // dynamic shared memory per CTA we allow ourselves (static use ~2 KB)

// Panel tiling: the rows of F^T (k, padded to kp) and of A (m, padded to mp)
// form one panel of Rp = kp + mp rows; the assets are cut into tiles of CH.
// One tiled copy, PE, feeds both matvec directions: a tile is Rp rows of CS
// elements (CH assets, then CS - CH zero pads), one contiguous block that one
// bulk copy moves into shared memory.  The pad makes the row stride an odd
// number of 4-byte words for 2- and 4-byte elements, so that the reduce pass
// (row groups reading the same assets of different rows) is free of shared-
// memory bank conflicts.
__host__ __device__ inline int tile_stride(int CH, int elem_bytes) { return CH + (elem_bytes == 2 ? 2 : 1); }

struct Tiling {
    int CH, CS, kp, mp, Rp, ntile;
    int vcap;             // single period: entries of v kept in shared memory (0: v in the workspace)
    int rep_glob;         // 1: per-period replicated arrays in the workspace (see rep_doubles)
};

__host__ __device__ inline Tiling make_tiling(int n, int k, int m, int CH, int elem_bytes) {
    Tiling t;
    t.CH = CH;
    t.CS = tile_stride(CH, elem_bytes);
    t.kp = (k + 7) / 8 * 8;
    t.mp = (m + 7) / 8 * 8;
    t.Rp = t.kp + t.mp;
    t.ntile = (n + CH - 1) / CH;
    t.vcap = 0;
    t.rep_glob = 0;
    return t;
}

// One instance as the solver kernel sees it (device memory).  All per-asset
// state arrays have row stride np (n rounded up to a multiple of 32).  Panels
// are stored as S (double, float or bfloat16) and multiplied in M (double or
// float); the iterate state and every elementwise update are FP64.
template <class M, class S>
struct Inst {
    int n, k, m, P, R, multi, np, omega_diag;
    int CH, CS, kp, mp, Rp, ntile; // panel tiling (see Tiling)
    int vcap;                  // > 0: v lives in shared memory (single period)
    int rep_glob;              // 1: yA, yAb, ax, u, ub of each CTA live in rep (workspace)
    double* rep;               // kMaxCluster slices of rep_doubles(P, k, m) doubles, or null
    const S* PE;          // ntile tiles of [Rp][CS]
    const double* Om;     // k x k, or k diagonal entries
    const M* alpha;       // P x np   (matvec precision: FP32 inputs stay exact)
    const M* Dp;          // P x np
    const double* Dmax;   // np       max over periods of D (for the Lipschitz bound)
    const M* c1;          // R x np   lambda2 * s
    const M* c2;          // R x np   lambda3 * q
    const double* w0;     // np
    const double* cen;    // np       risk centre: w_T (multi) or 0 (single)
    const double* alphaT; // np       alpha at t = T (multi) or unused
    const double* L;      // m
    const double* U;      // m
    double kappa, d;
    double GMV;
    // iterate storage (workspace)
    double *x, *x0, *xb, *xn, *v;      // P x np  (x, x0, xn: double-float pairs in the FP32/BF16
    double *yD, *yD0, *yDb, *yDn;      // R x np   modes once the setup is done; likewise yD, yD0, yDn)
    float* yDf;                        // R x np   FP32 copy of y_D (multi-period FP32 increments)
    const float* cenf;                 // np       FP32 copy of the centre
    const float2* w0f;                 // np       w0 as a double-float pair (FP32/BF16 modes)
    const float2* cen2;                // np       the centre as a double-float pair
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
    double beta_suff, beta_nec, beta_art;
    double step_fraction;
    double beta;
    int power_iters;
    int expire_first_wait;   // test hook (ff_options.test_expire_first_wait)
    int stall_checks;        // FP32/BF16 modes: checks without halving before FF_PRECISION (0 = off)
    int warm_start;          // 1: start from the output buffers (ff_options.warm_start)
    int panel_keep;          // 1: panel-tile copies carry an L2 evict_last policy
    int primal_weight;       // 1: adaptive primal weight at restarts (ff_options.primal_weight)
    int* queue;          // device counter of the next instance (zero at launch); teams take
                         // instances from it in table order
};

// Shared-memory bytes the solver kernel needs for these sizes and tiling.
size_t solver_smem_bytes(int P, int k, int m, int omega_diag, size_t matvec_size, int CH, int Rp, size_t panel_size,
                         int vcap, int rep_glob);

// Doubles of one CTA's slice of the replicated per-period arrays (rep_glob):
// yA (P m), yAb (Pr m), ax (P m), u (P k), ub (Pr k), Pr = P rounded up to
// whole chunks of kPC periods.
__host__ __device__ inline int rep_doubles(int P, int k, int m) {
    const int Pr = P <= 1 ? 1 : (P + kPC - 1) / kPC * kPC;
    const int d = 2 * P * m + Pr * m + P * k + Pr * k;
    return (d + 31) / 32 * 32;
}

// Largest tile width CH (256 down to 8) whose shared-memory layout fits, 0 if
// none does; for a single period it first tries to keep v (n entries, FP64)
// in shared memory as well and reports the capacity in *vcap (else 0); for
// many periods it moves the replicated per-period arrays to the workspace
// (*rep_glob = 1) when otherwise no tile of at least 32 assets fits.
int choose_tile(int P, int n, int k, int m, int omega_diag, size_t matvec_size, size_t panel_size, int* vcap,
                int* rep_glob);

// Joint primal prox variant (single period, FP64): workspace bytes (0 if an
// instance is not single-period or a size is invalid) and the launch of one
// CTA per instance; FF_ERR_UNSUPPORTED beyond 256 factors or exposure rows.
size_t joint_workspace_bytes(const ff_problem* probs, int count);
int joint_solve(const ff_problem* probs, int count, const Params& prm, void* ws, size_t ws_bytes, ff_result* res,
                void* const* w_out, void* const* yA_out, void* const* yD_out, cudaStream_t st, cudaError_t* cuda_err);

// Launch the team kernel over `count` instances (insts is a device array).
// G = CTAs per instance (cluster size), nteams = concurrent teams; single =
// every instance is single-period (the variant built for P = 1).
template <class M, class S>
cudaError_t launch_solver(const Inst<M, S>* insts, int count, const Params& prm, int G, int nteams,
                          size_t smem, bool single, cudaStream_t stream);

template <class M, class S>
cudaError_t max_teams(int G, size_t smem, bool single, int* out);

}  // namespace ff
