// Adjoint of the multi-period solve (Sec. 2.2, Eqs. 4-6): given the optimal
// trajectory x* = (w_1 .. w_{T-1}) and an upstream gradient g = dL/dx*, the
// vector-Jacobian products dL/d(alpha, F, D, s, q, w0, w_T) by implicit
// differentiation of the optimality conditions at x*.
//
// Scaled form (periods p = 0..P-1, P = T - 1; trades r = 0..P, R = T):
//   min sum_p [-alpha_p^T x_p + kappa (x_p - w_T)^T Sigma_p (x_p - w_T)]
//       + sum_r c1_r |z_r| + c2_r |z_r|^d,   z_r = x_r - x_{r-1},
// with x_{-1} = w0 and x_P = w_T, Sigma_p = F Omega F^T + diag(D_p), subject
// to the exposure rows L <= A x_p <= U and ||x_p||_1 <= 1 for every p.
//
// Active structure at x* (read from the forward outputs):
//   dead trade  : |yD_r| < c1_r (inside the spread dead zone), so x_r = x_{r-1};
//   zero holding: x_{p,i} == 0 (the l1 projection put it on its kink);
//   rows        : the l1 budget of period p when ||x_p||_1 = 1 (to rounding),
//                 exposure rows with a nonzero multiplier.
// Dead trades merge each asset's periods into runs; a run is FIXED when it
// touches w0 (dead first trade), w_T (dead last trade) or holds a zero, else it
// is a FREE group with one unknown.  With v the free-group values,
//   [H  E^T] [u ]   [S^T g]     H = S^T (blockdiag_p 2 kappa Sigma_p
//   [E   0 ] [nu] = [  0  ],          + Delta^T diag(h) Delta) S,
// h_r = c2_r d (d-1) |z_r|^(d-2) on live trades, E the active rows restricted
// to the free groups, and
//   dL/dtheta = u^T (-dr/dtheta) + nu^T (de/dtheta) + g^T dx_fixed/dtheta.
//
// GPU scheme: group-space vectors live in the period-major P x n layout at
// each group's first period.  H is applied matrix-free (one F^T pass and one
// F pass per application).  The system is solved by projected conjugate
// gradients with the residual update of Gould, Hribar and Nocedal (2001): the
// preconditioner M is the exact per-asset tridiagonal part (diag 2 kappa D +
// trade curvature), factored LDL^T along each asset's chain of groups; the
// projection onto null(E) uses C = E M^{-1} E^T, assembled once, factored by a
// Cholesky that drops dependent rows, and inverted explicitly so that each
// iteration applies it as a matrix-vector product.  The multipliers nu are the
// accumulated projection coefficients.  The whole computation is one
// cooperative launch over all instances of the batch: each step is a phase
// spread over the grid, phases are separated by a grid barrier whose waits are
// bounded, and the conjugate-gradient loop ends when every instance has
// stopped.  FP64 throughout.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "flashfolio.h"

namespace ff {
namespace {

constexpr int kRT = 256;              // threads of a block (8 warps)
constexpr int kNB = 32;               // columns of M^{-1} E^T per pass while C is assembled
constexpr int kMaxPcg = 600;          // iteration cap of the projected CG
constexpr double kPcgTol = 1e-11;     // stop when res^T M^{-1} res <= tol^2 of its first value
constexpr double kDropRel = 1e-12;    // Cholesky pivot / original diagonal below this: dependent row
constexpr double kZFloor = 1e-14;     // |z| used for the curvature of a live trade at 0

struct AdjM {
    int n, k, m, P, R, omega_diag, f64, rmax;
    const void *F, *Omega, *D, *alpha, *s, *q, *w0, *wT, *A;
    const void *w, *yA, *yD, *gw;
    void *dalpha, *dF, *dD, *ds, *dq, *dw0, *dwT;
    double kappa, lam2, lam3, d;
    // workspace (FP64 unless noted)
    int* gfirst;          // P n: first period of the holding's free group, -1 if fixed
    signed char* src;     // P n: -1 free, 0 fixed at zero, 1 fixed at w0, 2 fixed at w_T
    double* xfix;         // P n: value of a fixed holding (0 on free ones)
    double* hz;           // R n: trade curvature h_r (0 on dead trades)
    double* ldd;          // P n: LDL^T pivot of the chain, at group-first positions
    double* ldl;          // P n: LDL^T multiplier to the preceding linked group, at group-first positions
    double *u, *res, *zz, *pd, *hp;   // P n each: group-space CG vectors
    double *Uk, *Wk, *Uk2, *Wk2;      // P k each: F^T v per period and 2 kappa Omega F^T v
    int *rowp, *rowj;     // rmax: period and exposure row (-1 = budget) of each active row
    int* rowoff;          // P + 1: first active row of each period
    unsigned char* drop;  // rmax: row dropped as dependent
    double *C, *Ci, *Cd;  // rmax^2, rmax^2, rmax: E M^{-1} E^T (then its factor), its inverse, diagonal
    double* Z;            // P n kNB: columns of M^{-1} E^T while C is assembled
    double *ez, *wv, *nu; // rmax each
    double* part;         // n: per-asset partial sums of the CG inner products
    double* sc;           // [0] rz, [1] rz at the start, [2] step alpha, [3] beta
    int* flags;           // [0] active rows, [1] done, [2] iterations, [3] status
    int32_t* status_out;  // device or null
};

__device__ __forceinline__ double ldv(const void* p, size_t i, int f64) {
    return f64 ? ((const double*)p)[i] : (double)((const float*)p)[i];
}
__device__ __forceinline__ void stv(void* p, size_t i, double v, int f64) {
    if (!p) return;
    if (f64) ((double*)p)[i] = v;
    else ((float*)p)[i] = (float)v;
}
__device__ __forceinline__ double sgn(double x) { return x > 0 ? 1.0 : (x < 0 ? -1.0 : 0.0); }

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-wide reduction of one double per thread over kRT threads (sum or max)
template <bool kMax>
__device__ double block_reduce(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, v, o);
        v = kMax ? fmax(v, t) : v + t;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;   // the maxima taken here are of magnitudes (>= 0)
    for (int w = 0; w < kRT / 32; ++w) t = kMax ? fmax(t, red[w]) : t + red[w];
    __syncthreads();
    return t;
}

__device__ __forceinline__ bool dead_trade(const AdjM& I, int r, int i) {
    const size_t o = (size_t)r * I.n + i;
    return fabs(ldv(I.yD, o, I.f64)) < I.lam2 * ldv(I.s, o, I.f64);
}

// holding (p, i) as the adjoint sees it: the solver output on free holdings,
// the exact fixed value on fixed ones; w0 before the first period, w_T after the last
__device__ __forceinline__ double xe(const AdjM& I, int p, int i) {
    if (p < 0) return ldv(I.w0, i, I.f64);
    if (p >= I.P) return ldv(I.wT, i, I.f64);
    const size_t o = (size_t)p * I.n + i;
    return I.gfirst[o] >= 0 ? ldv(I.w, o, I.f64) : I.xfix[o];
}

// group-space vector v read at holding (p, i): the value of its free group, 0 if fixed or p outside 0..P-1
__device__ __forceinline__ double gv(const AdjM& I, const double* v, int p, int i) {
    if (p < 0 || p >= I.P) return 0.0;
    const int g = I.gfirst[(size_t)p * I.n + i];
    return g >= 0 ? v[(size_t)g * I.n + i] : 0.0;
}

// entry of active row (p, j) at the free holding (p, i): the holding's sign for
// the budget row (j < 0), else A_{j,i}
__device__ __forceinline__ double erow(const AdjM& I, int p, int j, int i) {
    if (j < 0) return sgn(ldv(I.w, (size_t)p * I.n + i, I.f64));
    return ldv(I.A, (size_t)j * I.n + i, I.f64);
}

// Solve M_i z = b on asset i's chain of free groups with the LDL^T factors
// (element (p, i) of b and z at index (p n + i) * stride + col; b may equal z).
__device__ void chain_solve(const AdjM& I, int i, const double* b, double* z, int stride, int col) {
    const int n = I.n, P = I.P;
    double yprev = 0;
    for (int p = 0; p < P; ++p) {
        const size_t o = (size_t)p * n + i;
        if (I.gfirst[o] != p) continue;
        const double y = b[o * stride + col] - I.ldl[o] * yprev;
        z[o * stride + col] = y;
        yprev = y;
    }
    double znext = 0, lnext = 0;
    for (int p = P - 1; p >= 0; --p) {
        const size_t o = (size_t)p * n + i;
        const int g = I.gfirst[o];
        if (g < 0) { znext = 0; lnext = 0; continue; }
        if (g != p) continue;
        const double zg = z[o * stride + col] / I.ldd[o] - lnext * znext;
        z[o * stride + col] = zg;
        znext = zg;
        lnext = I.ldl[o];
    }
}

// ---- grid-wide phases ------------------------------------------------------------
//
// The whole adjoint is one cooperative launch: every step below is a phase
// over all instances of the batch, and the phases are separated by a grid
// barrier.  A phase distributes its items over the grid in one of three ways:
// one item per thread (assets, (period, factor) pairs, columns), one item per
// warp (active rows, instances) or one item per block (instances).  Control
// flow that reaches a barrier is the same in every block: it depends only on
// values that all blocks read after the same barrier.

// Barrier state in the workspace (zeroed by the host before the launch).
struct GridSync {
    unsigned int arrive;   // blocks arrived at the current barrier
    unsigned int gen;      // barriers completed
    int expired;           // a block's wait passed its limit
    int pad;
};

constexpr long long kBarrierSpins = 1ll << 34;                   // polls of one wait
constexpr unsigned long long kBarrierNs = 60ull * 1000000000ull;  // or 60 s of device time

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long device_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every block arrives, the last one to arrive opens the next generation.  A
// wait ends after kBarrierSpins polls or kBarrierNs of device time: it then
// marks the launch expired and every block leaves at its next barrier.  A
// cooperative launch keeps all blocks resident, so a wait expires only when
// one phase runs longer than the limit (the one-block-per-instance Cholesky
// of a very large active row set) or the device stops scheduling blocks.
// Returns false once the launch expired.
__device__ bool grid_barrier(GridSync* gs) {
    __shared__ int ok_s;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = ld_acquire_u32(&gs->gen);
        int ok = 1;
        if (atomicAdd(&gs->arrive, 1u) == gridDim.x - 1) {
            atomicExch(&gs->arrive, 0u);
            st_release_u32(&gs->gen, g + 1);
        } else {
            const unsigned long long t0 = device_ns();
            for (long long s = 0; ld_acquire_u32(&gs->gen) == g; ++s) {
                if (s >= kBarrierSpins || ((s & 255) == 255 && device_ns() - t0 > kBarrierNs)) {
                    atomicExch(&gs->expired, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok && *(volatile int*)&gs->expired == 0;
    }
    __syncthreads();
    __threadfence();
    return ok_s != 0;
}

// fn(I, x) for every instance and every x < per(I) (one item per thread)
template <class Per, class Fn>
__device__ __forceinline__ void each_thread(const AdjM* insts, int count, int per_max, Per per, Fn fn) {
    const long long total = (long long)count * per_max, stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += stride) {
        const AdjM& I = insts[v / per_max];
        const int x = (int)(v % per_max);
        if (x < per(I)) fn(I, x);
    }
}

// fn(I, x, lane) for every instance and every x < per(I) (one item per warp)
template <class Per, class Fn>
__device__ __forceinline__ void each_warp(const AdjM* insts, int count, int per_max, Per per, Fn fn) {
    const int lane = threadIdx.x & 31;
    const long long total = (long long)count * per_max, stride = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long v = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < total; v += stride) {
        const AdjM& I = insts[v / per_max];
        const int x = (int)(v % per_max);
        if (x < per(I)) fn(I, x, lane);
    }
}

// ---- setup ------------------------------------------------------------------

// Per asset: runs of periods joined by dead trades, fixed or free; trade
// curvature; LDL^T of the chain's tridiagonal part.
__device__ void classify_at(const AdjM& I, int i) {
    const int n = I.n, P = I.P;
    int p = 0;
    while (p < P) {
        int q = p;
        while (q + 1 < P && dead_trade(I, q + 1, i)) ++q;   // trade q+1 joins periods q and q+1
        int code = -1;
        double fv = 0;
        if (p == 0 && dead_trade(I, 0, i)) { code = 1; fv = ldv(I.w0, i, I.f64); }
        if (code < 0 && q == P - 1 && dead_trade(I, P, i)) { code = 2; fv = ldv(I.wT, i, I.f64); }
        if (code < 0)
            for (int pp = p; pp <= q; ++pp)
                if (ldv(I.w, (size_t)pp * n + i, I.f64) == 0.0) { code = 0; fv = 0; break; }
        for (int pp = p; pp <= q; ++pp) {
            const size_t o = (size_t)pp * n + i;
            I.gfirst[o] = code < 0 ? p : -1;
            I.src[o] = (signed char)code;
            I.xfix[o] = code < 0 ? 0.0 : fv;
            I.ldd[o] = 0.0;
            I.ldl[o] = 0.0;
        }
        p = q + 1;
    }
    const double dexp = I.d;
    for (int r = 0; r <= P; ++r) {
        double h = 0;
        if (!dead_trade(I, r, i)) {
            const double c2 = I.lam3 * ldv(I.q, (size_t)r * n + i, I.f64);
            const double az = fmax(fabs(xe(I, r, i) - xe(I, r - 1, i)), kZFloor);
            h = c2 > 0 ? c2 * dexp * (dexp - 1.0) * pow(az, dexp - 2.0) : 0.0;
        }
        I.hz[(size_t)r * n + i] = h;
    }
    // tridiagonal part of H on the chain: diagonal sum_{p in g} 2 kappa D_p + h of
    // the two boundary trades; coupling -h to the group that ends just before
    double dprev = 0;
    int prev_end = -2;   // last period of the preceding free group
    p = 0;
    while (p < P) {
        const size_t o = (size_t)p * n + i;
        if (I.gfirst[o] < 0) { ++p; continue; }
        int q = p;
        while (q + 1 < P && I.gfirst[(size_t)(q + 1) * n + i] == p) ++q;
        double b = I.hz[o] + I.hz[(size_t)(q + 1) * n + i];
        for (int pp = p; pp <= q; ++pp) b += 2.0 * I.kappa * ldv(I.D, (size_t)pp * n + i, I.f64);
        double l = 0;
        if (prev_end == p - 1) {
            const double e = -I.hz[o];
            l = e / dprev;
            b -= l * e;
        }
        I.ldd[o] = b;
        I.ldl[o] = l;
        dprev = b;
        prev_end = q;
        p = q + 1;
    }
}

// Active rows of every period (one block per instance) and the zeroed multipliers.
__device__ void rows_block(const AdjM& I) {
    __shared__ double red[kRT / 32];
    __shared__ int r_s;
    const int tid = threadIdx.x, n = I.n, P = I.P, m = I.m;
    double ym = 0;
    for (int e = tid; e < P * m; e += kRT) ym = fmax(ym, fabs(ldv(I.yA, e, I.f64)));
    ym = block_reduce<true>(ym, red);
    // FP32 outputs carry their rounding into the l1 norm
    const double btol = I.f64 ? 1e-10 : 1e-6;
    if (tid == 0) r_s = 0;
    __syncthreads();
    for (int p = 0; p < P; ++p) {
        double l1 = 0;
        for (int i = tid; i < n; i += kRT) l1 += fabs(ldv(I.w, (size_t)p * n + i, I.f64));
        l1 = block_reduce<false>(l1, red);
        if (tid == 0) {
            int r = r_s;
            I.rowoff[p] = r;
            if (l1 >= 1.0 - btol) { I.rowp[r] = p; I.rowj[r] = -1; ++r; }
            for (int j = 0; j < m; ++j)
                if (ym > 0 && fabs(ldv(I.yA, (size_t)p * m + j, I.f64)) > 1e-12 * ym) {
                    I.rowp[r] = p;
                    I.rowj[r] = j;
                    ++r;
                }
            r_s = r;
        }
        __syncthreads();
    }
    if (tid == 0) {
        I.rowoff[P] = r_s;
        I.flags[0] = r_s;
        I.flags[1] = 0;
        I.flags[2] = 0;
        I.flags[3] = 0;
        I.sc[0] = I.sc[1] = I.sc[2] = I.sc[3] = 0.0;
    }
    for (int a = tid; a < I.rmax; a += kRT) { I.nu[a] = 0; I.wv[a] = 0; I.ez[a] = 0; I.drop[a] = 0; }
    __syncthreads();
}

// Columns c0 .. c0 + kNB - 1 of M^{-1} E^T (group space) for asset i.
__device__ void zcols_at(const AdjM& I, int i, int c0) {
    const int r = I.flags[0];
    if (c0 >= r) return;
    const int n = I.n, P = I.P;
    for (int cc = 0; cc < kNB && c0 + cc < r; ++cc) {
        const int c = c0 + cc;
        const int pc = I.rowp[c], jc = I.rowj[c];
        for (int p = 0; p < P; ++p) {
            const size_t o = (size_t)p * n + i;
            if (I.gfirst[o] == p) I.Z[o * kNB + cc] = 0.0;
        }
        const int g = I.gfirst[(size_t)pc * n + i];
        if (g < 0) continue;
        I.Z[((size_t)g * n + i) * kNB + cc] = erow(I, pc, jc, i);
        chain_solve(I, i, I.Z, I.Z, kNB, cc);
    }
}

// C[a][c] = E_a . (M^{-1} E^T)_c for row a and the columns c0 + lane.
__device__ void cfill_at(const AdjM& I, int a, int lane, int c0) {
    const int r = I.flags[0];
    const int c = c0 + lane;
    if (a >= r || c >= r) return;
    const int pa = I.rowp[a], ja = I.rowj[a], n = I.n;
    double acc = 0;
    for (int i = 0; i < n; ++i) {
        const int g = I.gfirst[(size_t)pa * n + i];
        if (g < 0) continue;
        acc += erow(I, pa, ja, i) * I.Z[((size_t)g * n + i) * kNB + lane];
    }
    I.C[(size_t)a * I.rmax + c] = acc;
}

// In-place Cholesky of C (one block per instance).  A row whose pivot falls to
// kDropRel of its original diagonal (or an empty row) is dependent on the rows
// before it: its row and column of the factor are cleared, its pivot set to 1,
// and it is marked dropped (its multiplier is 0).
__device__ void chol_block(const AdjM& I) {
    const int r = I.flags[0], ld = I.rmax;
    double* A = I.C;
    __shared__ int drop_s;
    for (int j = threadIdx.x; j < r; j += kRT) I.Cd[j] = A[(size_t)j * ld + j];
    __syncthreads();
    for (int j = 0; j < r; ++j) {
        if (threadIdx.x == 0) {
            const double piv = A[(size_t)j * ld + j];
            const int dr = !(piv > kDropRel * I.Cd[j]);
            drop_s = dr;
            I.drop[j] = (unsigned char)dr;
            A[(size_t)j * ld + j] = dr ? 1.0 : sqrt(piv);
        }
        __syncthreads();
        if (drop_s) {
            for (int i = j + 1 + threadIdx.x; i < r; i += kRT) A[(size_t)i * ld + j] = 0.0;
            for (int l = threadIdx.x; l < j; l += kRT) A[(size_t)j * ld + l] = 0.0;
            __syncthreads();
            continue;
        }
        const double ljj = A[(size_t)j * ld + j];
        for (int i = j + 1 + threadIdx.x; i < r; i += kRT) A[(size_t)i * ld + j] /= ljj;
        __syncthreads();
        const long long rem = r - j - 1;
        for (long long e = threadIdx.x; e < rem * rem; e += kRT) {
            const int ii = j + 1 + (int)(e / rem), l = j + 1 + (int)(e % rem);
            if (l <= ii) A[(size_t)ii * ld + l] -= A[(size_t)ii * ld + j] * A[(size_t)l * ld + j];
        }
        __syncthreads();
    }
}

// Column c of Ci = C^{-1} from the factor; the rows and columns of dropped rows are zero.
__device__ void inverse_at(const AdjM& I, int c) {
    const int r = I.flags[0], ld = I.rmax;
    const double* L = I.C;
    double* X = I.Ci;
    for (int i = 0; i < r; ++i) {
        double v = 0;
        if (i == c) v = 1.0;
        if (i > c)
            for (int l = c; l < i; ++l) v -= L[(size_t)i * ld + l] * X[(size_t)l * ld + c];
        X[(size_t)i * ld + c] = i < c ? 0.0 : v / L[(size_t)i * ld + i];
    }
    for (int i = r - 1; i >= 0; --i) {
        double v = X[(size_t)i * ld + c];
        for (int l = i + 1; l < r; ++l) v -= L[(size_t)l * ld + i] * X[(size_t)l * ld + c];
        X[(size_t)i * ld + c] = v / L[(size_t)i * ld + i];
    }
    const bool dc = I.drop[c] != 0;
    for (int i = 0; i < r; ++i)
        if (dc || I.drop[i]) X[(size_t)i * ld + c] = 0.0;
}

// ---- projected conjugate gradients ---------------------------------------------

// res = -S^T g, u = pd = 0, zz = M^{-1} res for asset i
__device__ void pcg_init_at(const AdjM& I, int i) {
    const int n = I.n, P = I.P;
    for (int p = 0; p < P; ++p) {
        const size_t o = (size_t)p * n + i;
        const int g = I.gfirst[o];
        if (g < 0) continue;
        const double gw = ldv(I.gw, o, I.f64);
        if (g == p) {
            I.res[o] = -gw;
            I.u[o] = 0.0;
            I.pd[o] = 0.0;
            I.hp[o] = 0.0;
        } else {
            I.res[(size_t)g * n + i] -= gw;
        }
    }
    chain_solve(I, i, I.res, I.zz, 1, 0);
}

// ez[a] = E_a zz (one warp per active row)
__device__ void ez_at(const AdjM& I, int a, int lane) {
    if (I.flags[1] || a >= I.flags[0]) return;
    const int pa = I.rowp[a], ja = I.rowj[a], n = I.n;
    double acc = 0;
    for (int i = lane; i < n; i += 32) {
        const int g = I.gfirst[(size_t)pa * n + i];
        if (g >= 0) acc += erow(I, pa, ja, i) * I.zz[(size_t)g * n + i];
    }
    acc = warp_sum(acc);
    if (lane == 0) I.ez[a] = acc;
}

// w[a] = (C^{-1} ez)_a; nu[a] -= w[a] (one warp per active row)
__device__ void w_at(const AdjM& I, int a, int lane) {
    const int r = I.flags[0];
    if (I.flags[1] || a >= r) return;
    double acc = 0;
    for (int c = lane; c < r; c += 32) acc += I.Ci[(size_t)a * I.rmax + c] * I.ez[c];
    acc = warp_sum(acc);
    if (lane == 0) {
        I.wv[a] = acc;
        I.nu[a] -= acc;
    }
}

// res -= E^T w, zz = M^{-1} res, part = res . zz for asset i
__device__ void update_res_at(const AdjM& I, int i) {
    if (I.flags[1]) return;
    const int n = I.n, P = I.P;
    for (int p = 0; p < P; ++p) {
        const size_t o = (size_t)p * n + i;
        const int g = I.gfirst[o];
        if (g < 0) continue;
        double qv = 0;
        for (int a = I.rowoff[p]; a < I.rowoff[p + 1]; ++a) qv += I.wv[a] * erow(I, p, I.rowj[a], i);
        I.res[(size_t)g * n + i] -= qv;
    }
    chain_solve(I, i, I.res, I.zz, 1, 0);
    double s = 0;
    for (int p = 0; p < P; ++p) {
        const size_t o = (size_t)p * n + i;
        if (I.gfirst[o] == p) s += I.res[o] * I.zz[o];
    }
    I.part[i] = s;
}

// rz = sum(part): first value (init), else beta and the stopping test (one warp per instance)
__device__ void rz_at(const AdjM& I, int lane, int init) {
    if (I.flags[1]) return;
    double s = 0;
    for (int i = lane; i < I.n; i += 32) s += I.part[i];
    s = warp_sum(s);
    if (lane != 0) return;
    if (!isfinite(s)) { I.flags[3] = 4; I.flags[1] = 1; return; }
    if (init) {
        I.sc[0] = s;
        I.sc[1] = s;
        I.sc[3] = 0.0;
        if (!(s > 0)) I.flags[1] = 1;   // the projected gradient is zero: u = 0
        return;
    }
    I.flags[2] += 1;
    I.sc[3] = s / I.sc[0];
    I.sc[0] = s;
    if (!(s > kPcgTol * kPcgTol * I.sc[1])) I.flags[1] = 1;
    else if (I.flags[2] >= kMaxPcg) { I.flags[3] = 3; I.flags[1] = 1; }
}

// pd = -zz + beta pd for asset i
__device__ void pdir_at(const AdjM& I, int i) {
    if (I.flags[1]) return;
    const double beta = I.sc[3];
    for (int p = 0; p < I.P; ++p) {
        const size_t o = (size_t)p * I.n + i;
        if (I.gfirst[o] == p) I.pd[o] = -I.zz[o] + beta * I.pd[o];
    }
}

// Uk[p][j] = sum_i v(p, i) F_{i,j} for v = pd (which 0), u (which 1) or, into
// Uk2, the centred holdings x_p - w_T (which 2); e = p k + j.
__device__ void prodF_at(const AdjM& I, int e, int which) {
    if (which == 0 && I.flags[1]) return;
    const int n = I.n, k = I.k;
    const int p = e / k, j = e % k;
    double acc = 0;
    if (which == 2) {
        for (int i = 0; i < n; ++i)
            acc += (xe(I, p, i) - ldv(I.wT, i, I.f64)) * ldv(I.F, (size_t)i * k + j, I.f64);
        I.Uk2[e] = acc;
    } else {
        const double* v = which == 0 ? I.pd : I.u;
        for (int i = 0; i < n; ++i) {
            const int g = I.gfirst[(size_t)p * n + i];
            if (g >= 0) acc += v[(size_t)g * n + i] * ldv(I.F, (size_t)i * k + j, I.f64);
        }
        I.Uk[e] = acc;
    }
}

// W[p] = 2 kappa Omega U[p] for (Uk -> Wk) (which 0) or (Uk2 -> Wk2) (which 1); e = p k + j
__device__ void omega_at(const AdjM& I, int e, int which, int in_pcg) {
    if (in_pcg && I.flags[1]) return;
    const int k = I.k;
    const int p = e / k, j = e % k;
    const double* U = which == 0 ? I.Uk : I.Uk2;
    double* W = which == 0 ? I.Wk : I.Wk2;
    double acc;
    if (I.omega_diag) {
        acc = ldv(I.Omega, j, I.f64) * U[e];
    } else {
        acc = 0;
        for (int l = 0; l < k; ++l) acc += ldv(I.Omega, (size_t)j * k + l, I.f64) * U[(size_t)p * k + l];
    }
    W[e] = 2.0 * I.kappa * acc;
}

// hp = H pd (group space) and part = pd . hp for asset i
__device__ void hp_at(const AdjM& I, int i) {
    if (I.flags[1]) return;
    const int n = I.n, P = I.P, k = I.k;
    double vprev = 0, vcur = gv(I, I.pd, 0, i);
    for (int p = 0; p < P; ++p) {
        const double vnext = gv(I, I.pd, p + 1, i);
        const size_t o = (size_t)p * n + i;
        const int g = I.gfirst[o];
        if (g >= 0) {
            double y = 2.0 * I.kappa * ldv(I.D, o, I.f64) * vcur;
            for (int j = 0; j < k; ++j) y += ldv(I.F, (size_t)i * k + j, I.f64) * I.Wk[(size_t)p * k + j];
            y += I.hz[o] * (vcur - vprev) - I.hz[(size_t)(p + 1) * n + i] * (vnext - vcur);
            if (g == p) I.hp[o] = y;
            else I.hp[(size_t)g * n + i] += y;
        }
        vprev = vcur;
        vcur = vnext;
    }
    double s = 0;
    for (int p = 0; p < P; ++p) {
        const size_t o = (size_t)p * n + i;
        if (I.gfirst[o] == p) s += I.pd[o] * I.hp[o];
    }
    I.part[i] = s;
}

// alpha = rz / (pd . H pd) (one warp per instance)
__device__ void alpha_at(const AdjM& I, int lane) {
    if (I.flags[1]) return;
    double s = 0;
    for (int i = lane; i < I.n; i += 32) s += I.part[i];
    s = warp_sum(s);
    if (lane != 0) return;
    if (!(s > 0) || !isfinite(s)) { I.flags[3] = 4; I.flags[1] = 1; return; }
    I.sc[2] = I.sc[0] / s;
}

// u += alpha pd, res += alpha hp, zz = M^{-1} res for asset i
__device__ void step_at(const AdjM& I, int i) {
    if (I.flags[1]) return;
    const double al = I.sc[2];
    for (int p = 0; p < I.P; ++p) {
        const size_t o = (size_t)p * I.n + i;
        if (I.gfirst[o] != p) continue;
        I.u[o] += al * I.pd[o];
        I.res[o] += al * I.hp[o];
    }
    chain_solve(I, i, I.res, I.zz, 1, 0);
}

// ---- assembly -------------------------------------------------------------------

// Asset i: d alpha, d D (periods), d s, d q (trades), d w0, d w_T.
__device__ void grad_asset_at(const AdjM& I, int i) {
    const int n = I.n, P = I.P, k = I.k, f64 = I.f64;
    const double kap = I.kappa, dexp = I.d;
    const double wTi = ldv(I.wT, i, f64);
    double dw0 = 0, dwT = 0;
    // trades: d s, d q and the h_r (u_r - u_{r-1}) terms
    for (int r = 0; r <= P; ++r) {
        const size_t o = (size_t)r * n + i;
        const bool live = !dead_trade(I, r, i);
        const double z = xe(I, r, i) - xe(I, r - 1, i);
        const double duz = gv(I, I.u, r, i) - gv(I, I.u, r - 1, i);
        const double sz = sgn(z);
        stv(I.ds, o, live ? -I.lam2 * sz * duz : 0.0, f64);
        stv(I.dq, o, live ? -I.lam3 * dexp * pow(fabs(z), dexp - 1.0) * sz * duz : 0.0, f64);
        const double hd = I.hz[o] * duz;
        if (r == 0) dw0 += hd;
        if (r == P) dwT -= hd;
    }
    for (int p = 0; p < P; ++p) {
        const size_t o = (size_t)p * n + i;
        const double up = gv(I, I.u, p, i);
        const double dX = xe(I, p, i) - wTi;
        double y = 2.0 * kap * ldv(I.D, o, f64) * up;
        for (int j = 0; j < k; ++j) y += ldv(I.F, (size_t)i * k + j, f64) * I.Wk[(size_t)p * k + j];
        stv(I.dalpha, o, up, f64);
        stv(I.dD, o, -2.0 * kap * dX * up, f64);
        dwT += y;
        const int sc = I.src[o];
        if (sc == 1 || sc == 2) {
            const double hl = I.hz[o] * (gv(I, I.u, p, i) - gv(I, I.u, p - 1, i));
            const double hr = I.hz[(size_t)(p + 1) * n + i] * (gv(I, I.u, p + 1, i) - gv(I, I.u, p, i));
            double cf = ldv(I.gw, o, f64) - y - (hl - hr);
            const double sx = sgn(I.xfix[o]);
            for (int a = I.rowoff[p]; a < I.rowoff[p + 1]; ++a) {
                const int j = I.rowj[a];
                cf -= I.nu[a] * (j < 0 ? sx : ldv(I.A, (size_t)j * n + i, f64));
            }
            if (sc == 1) dw0 += cf;
            else dwT += cf;
        }
    }
    // the last row of alpha and D enters only a constant
    stv(I.dalpha, (size_t)P * n + i, 0.0, f64);
    stv(I.dD, (size_t)P * n + i, 0.0, f64);
    stv(I.dw0, i, dw0, f64);
    stv(I.dwT, i, dwT, f64);
}

// d F[i][j] = -sum_p (u_{p,i} Wk2[p][j] + (x_{p,i} - w_T,i) Wk[p][j]); e = i k + j
__device__ void grad_F_at(const AdjM& I, int e) {
    if (!I.dF) return;
    const int k = I.k;
    const int i = e / k, j = e % k;
    const double wTi = ldv(I.wT, i, I.f64);
    double acc = 0;
    for (int p = 0; p < I.P; ++p)
        acc += gv(I, I.u, p, i) * I.Wk2[(size_t)p * k + j] + (xe(I, p, i) - wTi) * I.Wk[(size_t)p * k + j];
    stv(I.dF, e, -acc, I.f64);
}

// Largest size of the batch for each item space of the phases.
struct Extents {
    int n;      // assets
    int rows;   // rows_max = (T-1)(m+1)
    int pk;     // (T-1) k
    int nk;     // n k
};

// The adjoint of every instance: setup, the projected conjugate gradients
// (converged instances take no further part; the loop ends when every
// instance has stopped) and the assembly of the products.
__global__ void __launch_bounds__(kRT) adjm_kernel(const AdjM* __restrict__ insts, int count, Extents ex,
                                                   GridSync* gs) {
    auto nA = [](const AdjM& I) { return I.n; };
    auto nR = [](const AdjM& I) { return I.rmax; };
    auto nPK = [](const AdjM& I) { return I.P * I.k; };
    auto nNK = [](const AdjM& I) { return I.n * I.k; };
    auto one = [](const AdjM&) { return 1; };
    __shared__ int flag_s;

    each_thread(insts, count, ex.n, nA, [](const AdjM& I, int i) { classify_at(I, i); });
    if (!grid_barrier(gs)) goto expired;
    for (int t = blockIdx.x; t < count; t += gridDim.x) rows_block(insts[t]);
    if (!grid_barrier(gs)) goto expired;
    {
        // the passes over the columns of M^{-1} E^T cover the largest active row count
        int rmax_act = 0;
        for (int t = 0; t < count; ++t) rmax_act = max(rmax_act, *(volatile int*)&insts[t].flags[0]);
        for (int c0 = 0; c0 < rmax_act; c0 += kNB) {
            each_thread(insts, count, ex.n, nA, [c0](const AdjM& I, int i) { zcols_at(I, i, c0); });
            if (!grid_barrier(gs)) goto expired;
            each_warp(insts, count, ex.rows, nR, [c0](const AdjM& I, int a, int lane) { cfill_at(I, a, lane, c0); });
            if (!grid_barrier(gs)) goto expired;
        }
    }
    for (int t = blockIdx.x; t < count; t += gridDim.x) chol_block(insts[t]);
    if (!grid_barrier(gs)) goto expired;
    each_thread(insts, count, ex.rows, nR, [](const AdjM& I, int c) { if (c < I.flags[0]) inverse_at(I, c); });
    if (!grid_barrier(gs)) goto expired;

    // first projection: res = -S^T g, then the component in null(E)
    each_thread(insts, count, ex.n, nA, [](const AdjM& I, int i) { pcg_init_at(I, i); });
    if (!grid_barrier(gs)) goto expired;
    each_warp(insts, count, ex.rows, nR, [](const AdjM& I, int a, int lane) { ez_at(I, a, lane); });
    if (!grid_barrier(gs)) goto expired;
    each_warp(insts, count, ex.rows, nR, [](const AdjM& I, int a, int lane) { w_at(I, a, lane); });
    if (!grid_barrier(gs)) goto expired;
    each_thread(insts, count, ex.n, nA, [](const AdjM& I, int i) { update_res_at(I, i); });
    if (!grid_barrier(gs)) goto expired;
    each_warp(insts, count, 1, one, [](const AdjM& I, int, int lane) { rz_at(I, lane, 1); });
    if (!grid_barrier(gs)) goto expired;
    each_thread(insts, count, ex.n, nA, [](const AdjM& I, int i) { pdir_at(I, i); });
    if (!grid_barrier(gs)) goto expired;

    for (int it = 0; it < kMaxPcg; ++it) {
        // every block reads the same stop flags here: they change only in the
        // alpha and rz phases, each followed by a barrier
        if (threadIdx.x == 0) {
            int live = 0;
            for (int t = 0; t < count && !live; ++t) live = *(volatile int*)&insts[t].flags[1] == 0;
            flag_s = live;
        }
        __syncthreads();
        const int live = flag_s;
        __syncthreads();
        if (!live) break;
        each_thread(insts, count, ex.pk, nPK, [](const AdjM& I, int e) { prodF_at(I, e, 0); });
        if (!grid_barrier(gs)) goto expired;
        each_thread(insts, count, ex.pk, nPK, [](const AdjM& I, int e) { omega_at(I, e, 0, 1); });
        if (!grid_barrier(gs)) goto expired;
        each_thread(insts, count, ex.n, nA, [](const AdjM& I, int i) { hp_at(I, i); });
        if (!grid_barrier(gs)) goto expired;
        each_warp(insts, count, 1, one, [](const AdjM& I, int, int lane) { alpha_at(I, lane); });
        if (!grid_barrier(gs)) goto expired;
        each_thread(insts, count, ex.n, nA, [](const AdjM& I, int i) { step_at(I, i); });
        if (!grid_barrier(gs)) goto expired;
        each_warp(insts, count, ex.rows, nR, [](const AdjM& I, int a, int lane) { ez_at(I, a, lane); });
        if (!grid_barrier(gs)) goto expired;
        each_warp(insts, count, ex.rows, nR, [](const AdjM& I, int a, int lane) { w_at(I, a, lane); });
        if (!grid_barrier(gs)) goto expired;
        each_thread(insts, count, ex.n, nA, [](const AdjM& I, int i) { update_res_at(I, i); });
        if (!grid_barrier(gs)) goto expired;
        each_warp(insts, count, 1, one, [](const AdjM& I, int, int lane) { rz_at(I, lane, 0); });
        if (!grid_barrier(gs)) goto expired;
        each_thread(insts, count, ex.n, nA, [](const AdjM& I, int i) { pdir_at(I, i); });
        if (!grid_barrier(gs)) goto expired;
    }

    // assembly: F^T u and F^T (x - w_T), their Omega products, the gradients
    each_thread(insts, count, ex.pk, nPK, [](const AdjM& I, int e) { prodF_at(I, e, 1); prodF_at(I, e, 2); });
    if (!grid_barrier(gs)) goto expired;
    each_thread(insts, count, ex.pk, nPK, [](const AdjM& I, int e) { omega_at(I, e, 0, 0); omega_at(I, e, 1, 0); });
    if (!grid_barrier(gs)) goto expired;
    each_thread(insts, count, ex.n, nA, [](const AdjM& I, int i) { grad_asset_at(I, i); });
    each_thread(insts, count, ex.nk, nNK, [](const AdjM& I, int e) { grad_F_at(I, e); });
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x)
        if (insts[t].status_out) *insts[t].status_out = insts[t].flags[3];
    return;

expired:
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        insts[t].flags[3] = 5;
        insts[t].flags[1] = 1;
        if (insts[t].status_out) *insts[t].status_out = 5;
    }
}

inline size_t a256(size_t x) { return (x + 255) / 256 * 256; }

size_t rows_max(int m, int T) { return (size_t)(T - 1) * (size_t)(m + 1); }

size_t adjm_bytes(int n, int k, int m, int T) {
    const size_t P = (size_t)T - 1, R = (size_t)T, PN = P * (size_t)n, rmax = rows_max(m, T);
    size_t b = 0;
    b += a256(PN * 4) + a256(PN) + a256(PN * 8) + a256(R * n * 8) + 2 * a256(PN * 8);   // gfirst src xfix hz ldd ldl
    b += 5 * a256(PN * 8);                                                              // u res zz pd hp
    b += 4 * a256(P * k * 8);                                                           // Uk Wk Uk2 Wk2
    b += 2 * a256(rmax * 4) + a256((P + 1) * 4) + a256(rmax);                           // rowp rowj rowoff drop
    b += 2 * a256(rmax * rmax * 8) + a256(rmax * 8);                                    // C Ci Cd
    b += a256(PN * kNB * 8);                                                            // Z
    b += 3 * a256(rmax * 8) + a256((size_t)n * 8) + a256(8 * 8) + a256(8 * 4);          // ez wv nu part sc flags
    return b;
}

bool valid_multi(const ff_problem* p, const void* w, const void* yA, const void* yD, const void* grad_w,
                 const ff_grads* out) {
    if (!p || p->T < 2 || !w || !yD || !grad_w || !out) return false;
    if (p->n < 1 || p->k < 1 || p->m < 0 || (p->m > 0 && (!yA || !p->A))) return false;
    if (p->dtype != FF_F64 && p->dtype != FF_F32) return false;
    if (!p->F || !p->Omega || !p->D || !p->alpha || !p->s || !p->q || !p->w0 || !p->wT) return false;
    if (!(p->GMV > 0) || !(p->lambda1 > 0) || !(p->d > 1.0 && p->d <= 2.0)) return false;
    if (!(p->lambda2 >= 0) || !(p->lambda3 >= 0)) return false;
    return true;
}

AdjM carve_multi(const ff_problem* p, const void* w, const void* yA, const void* yD, const void* grad_w,
                 const ff_grads* out, unsigned char*& cur, int32_t* status_out) {
    AdjM I;
    memset(&I, 0, sizeof(I));
    I.n = p->n; I.k = p->k; I.m = p->m; I.P = p->T - 1; I.R = p->T;
    I.omega_diag = p->omega_diag ? 1 : 0; I.f64 = p->dtype == FF_F64;
    I.rmax = (int)rows_max(p->m, p->T);
    I.F = p->F; I.Omega = p->Omega; I.D = p->D; I.alpha = p->alpha; I.s = p->s; I.q = p->q;
    I.w0 = p->w0; I.wT = p->wT; I.A = p->A;
    I.w = w; I.yA = yA; I.yD = yD; I.gw = grad_w;
    I.dalpha = out->alpha; I.dF = out->F; I.dD = out->D; I.ds = out->s; I.dq = out->q;
    I.dw0 = out->w0; I.dwT = out->wT;
    I.kappa = p->lambda1 * p->GMV; I.lam2 = p->lambda2; I.lam3 = p->lambda3; I.d = p->d;
    auto take = [&](size_t bytes) { unsigned char* r = cur; cur += a256(bytes); return (void*)r; };
    const size_t P = (size_t)I.P, R = (size_t)I.R, n = (size_t)I.n, k = (size_t)I.k, PN = P * n;
    const size_t rmax = (size_t)I.rmax;
    I.gfirst = (int*)take(PN * 4);
    I.src = (signed char*)take(PN);
    I.xfix = (double*)take(PN * 8);
    I.hz = (double*)take(R * n * 8);
    I.ldd = (double*)take(PN * 8);
    I.ldl = (double*)take(PN * 8);
    I.u = (double*)take(PN * 8);
    I.res = (double*)take(PN * 8);
    I.zz = (double*)take(PN * 8);
    I.pd = (double*)take(PN * 8);
    I.hp = (double*)take(PN * 8);
    I.Uk = (double*)take(P * k * 8);
    I.Wk = (double*)take(P * k * 8);
    I.Uk2 = (double*)take(P * k * 8);
    I.Wk2 = (double*)take(P * k * 8);
    I.rowp = (int*)take(rmax * 4);
    I.rowj = (int*)take(rmax * 4);
    I.rowoff = (int*)take((P + 1) * 4);
    I.drop = (unsigned char*)take(rmax);
    I.C = (double*)take(rmax * rmax * 8);
    I.Ci = (double*)take(rmax * rmax * 8);
    I.Cd = (double*)take(rmax * 8);
    I.Z = (double*)take(PN * kNB * 8);
    I.ez = (double*)take(rmax * 8);
    I.wv = (double*)take(rmax * 8);
    I.nu = (double*)take(rmax * 8);
    I.part = (double*)take(n * 8);
    I.sc = (double*)take(8 * 8);
    I.flags = (int*)take(8 * 4);
    I.status_out = status_out;
    return I;
}

}  // namespace
}  // namespace ff

extern "C" {

size_t ff_backward_multi_workspace_size(const ff_problem* probs, int count) {
    if (!probs || count < 1) return 0;
    size_t b = ff::a256((size_t)count * sizeof(ff::AdjM)) + ff::a256(sizeof(ff::GridSync));
    for (int t = 0; t < count; ++t) {
        const ff_problem* p = &probs[t];
        if (p->T < 2 || p->n < 1 || p->k < 1 || p->m < 0) return 0;
        b += ff::adjm_bytes(p->n, p->k, p->m, p->T);
    }
    return b;
}

int ff_backward_multi_batch(const ff_problem* probs, int count, const void* const* w, const void* const* yA,
                            const void* const* yD, const void* const* grad_w, const ff_grads* out, void* ws,
                            size_t ws_bytes, int32_t* status_dev, void* stream) {
    if (!probs || count < 1 || count > 65535 || !w || !yD || !grad_w || !out) return FF_ERR_INVALID_ARG;
    int nmax = 0, rmax = 0, pkmax = 0, nkmax = 0;
    for (int t = 0; t < count; ++t) {
        const ff_problem* p = &probs[t];
        if (!ff::valid_multi(p, w[t], yA ? yA[t] : nullptr, yD[t], grad_w[t], &out[t])) return FF_ERR_INVALID_ARG;
        const size_t rm = ff::rows_max(p->m, p->T);
        const size_t pk = (size_t)(p->T - 1) * p->k, nk = (size_t)p->n * p->k;
        if (rm > (1u << 20) || pk > (1u << 30) || nk > (1u << 30) || (size_t)p->n * (p->T - 1) > (1u << 30))
            return FF_ERR_UNSUPPORTED;
        nmax = std::max(nmax, p->n);
        rmax = std::max(rmax, (int)rm);
        pkmax = std::max(pkmax, (int)pk);
        nkmax = std::max(nkmax, (int)nk);
    }
    const size_t need = ff_backward_multi_workspace_size(probs, count);
    if (!ws || ((uintptr_t)ws % 256) != 0 || ws_bytes < need) return FF_ERR_WORKSPACE;
    int dev = 0, coop = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ff::adjm_kernel, ff::kRT, 0) != cudaSuccess)
        return FF_ERR_CUDA;
    if (!coop || occ < 1 || sms < 1) return FF_ERR_UNSUPPORTED;
    unsigned char* base = (unsigned char*)ws;
    ff::GridSync* gs = (ff::GridSync*)(base + ff::a256((size_t)count * sizeof(ff::AdjM)));
    unsigned char* cur = (unsigned char*)gs + ff::a256(sizeof(ff::GridSync));
    std::vector<ff::AdjM> table(count);
    for (int t = 0; t < count; ++t)
        table[t] = ff::carve_multi(&probs[t], w[t], yA ? yA[t] : nullptr, yD[t], grad_w[t], &out[t], cur,
                                   status_dev ? status_dev + t : nullptr);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(base, table.data(), (size_t)count * sizeof(ff::AdjM), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemsetAsync(gs, 0, sizeof(ff::GridSync), st) != cudaSuccess)
        return FF_ERR_CUDA;
    // one block per SM, more (up to the occupancy, at most 4) when the
    // per-asset phases have more assets than one block per SM has threads
    const long long items = (long long)count * nmax;
    int per_sm = (int)std::min<long long>(4, (items + (long long)sms * ff::kRT - 1) / ((long long)sms * ff::kRT));
    per_sm = std::max(1, std::min(per_sm, occ));
    const ff::AdjM* T = (const ff::AdjM*)base;
    ff::Extents ex{nmax, rmax, pkmax, nkmax};
    void* args[] = {(void*)&T, (void*)&count, (void*)&ex, (void*)&gs};
    if (cudaLaunchCooperativeKernel((const void*)ff::adjm_kernel, dim3(sms * per_sm), dim3(ff::kRT), args, 0, st) !=
        cudaSuccess)
        return FF_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return FF_ERR_CUDA;
    return FF_OK;
}

}  // extern "C"
