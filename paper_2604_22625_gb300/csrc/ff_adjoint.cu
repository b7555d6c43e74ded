// Adjoint of the single-period solve (Sec. 2.1, Eqs. 1-3): given the optimal
// portfolio w* and an upstream gradient g = dL/dw*, the vector-Jacobian
// products dL/d(alpha, F, D, s, q, w0) by implicit differentiation of the
// optimality conditions at w*.
//
// In the scaled form  min -alpha^T x + kappa x^T Sigma x + sum_i c1_i |z_i| +
// c2_i |z_i|^d,  z = x - w0,  Sigma = F Omega F^T + diag(D), kappa = lambda1
// GMV, c1 = lambda2 s, c2 = lambda3 q, subject to the active exposure rows and
// the l1 budget, each asset is either
//   zero  : x_i = 0 (the l1 projection put it on its kink),
//   dead  : x_i = w0_i (|yD_i| < c1_i: inside the spread dead zone),
//   free  : both kinks inactive; the objective is smooth in x_i.
// With those fixed, the free block S satisfies  r_S(x, theta) + E^T nu = 0,
// E x_S = e  (E: sign row of the active budget and the active rows of A), so
//   [H  E^T] [u ]   [g_S]      H = diag(h) + 2 kappa F_S Omega F_S^T,
//   [E   0 ] [nu] = [ 0 ],     h_i = 2 kappa D_i + c2_i d (d-1) |z_i|^(d-2),
// and dL/dtheta = u^T (-dr_S/dtheta) + nu^T (de/dtheta) + g_fixed^T dx_fixed/dtheta.
// H^{-1} by Woodbury through the k x k matrix M = (2 kappa Omega)^{-1} +
// F_S^T diag(1/h) F_S, the constraints by the Schur complement
// E H^{-1} E^T.  One CTA per instance, FP64 throughout (a small fraction of
// the forward solve's work).
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ff_internal.cuh"

namespace ff {
namespace {

constexpr int kAdjThreads = 256;

struct AdjInst {
    int n, k, m, omega_diag, in_f64;
    const void *F, *Omega, *D, *alpha, *s, *q, *w0, *A;
    const void *w, *yA, *yD, *gw;
    void *dalpha, *dF, *dD, *ds, *dq, *dw0;
    double kappa, lam2, lam3, d;
    // workspace (FP64 unless noted)
    double* invh;        // n: 1/h_i on free assets, 0 on fixed ones
    signed char* cls;    // n: 0 free, 1 zero holding, 2 dead trade
    double* u;           // n: adjoint of the free block (0 elsewhere)
    int* rows;           // m + 1: active constraints, -1 = budget, j = exposure row j
    double* M;           // k x k
    double* Oi;          // k x k: (2 kappa Omega)^{-1} (full Omega only)
    double* W;           // k x (m + 2): F_S^T diag(1/h) [g, E^T]
    double* Sc;          // (m + 1) x (m + 1): E diag(1/h) E^T, then the Schur complement
    double* vr;          // 4 (m + 2): E diag(1/h) g, nu, scratch
    double* vk;          // 6 k: F^T x, F^T u, Omega F^T x, Omega F^T u, t, scratch
    int* flags;          // [0] number of active constraints, [1] status
    int32_t* status_out; // device or null: the instance's status
};

__device__ __forceinline__ double ld(const void* p, size_t i, int f64) {
    return f64 ? ((const double*)p)[i] : (double)((const float*)p)[i];
}
__device__ __forceinline__ void st(void* p, size_t i, double v, int f64) {
    if (!p) return;
    if (f64) ((double*)p)[i] = v;
    else ((float*)p)[i] = (float)v;
}

// block-wide sum of one double per thread (every thread receives the total)
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0;
    for (int w = 0; w < kAdjThreads / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

// In-place Cholesky A = L L^T of the leading N x N block (row-major with
// leading dimension lda, lower triangle used); returns false when a pivot is
// not positive.  Right-looking, all threads of the CTA share the trailing update.
__device__ bool cholesky(double* A, int N, int lda, double* flag) {
    for (int j = 0; j < N; ++j) {
        if (threadIdx.x == 0) {
            const double piv = A[(size_t)j * lda + j];
            *flag = piv;
            A[(size_t)j * lda + j] = piv > 0 ? sqrt(piv) : 1.0;
        }
        __syncthreads();
        if (!(*flag > 0)) return false;
        const double ljj = A[(size_t)j * lda + j];
        for (int i = j + 1 + threadIdx.x; i < N; i += kAdjThreads) A[(size_t)i * lda + j] /= ljj;
        __syncthreads();
        const int rem = N - j - 1;
        for (int e = threadIdx.x; e < rem * rem; e += kAdjThreads) {
            const int i = j + 1 + e / rem, l = j + 1 + e % rem;
            if (l <= i) A[(size_t)i * lda + l] -= A[(size_t)i * lda + j] * A[(size_t)l * lda + j];
        }
        __syncthreads();
    }
    return true;
}

// Solve L L^T X = B for NB right-hand sides stored as columns of B (N x NB,
// leading dimension ldb); thread c handles column c.
__device__ void chol_solve(const double* L, int N, int lda, double* B, int NB, int ldb) {
    for (int c = threadIdx.x; c < NB; c += kAdjThreads) {
        for (int i = 0; i < N; ++i) {
            double v = B[(size_t)i * ldb + c];
            for (int l = 0; l < i; ++l) v -= L[(size_t)i * lda + l] * B[(size_t)l * ldb + c];
            B[(size_t)i * ldb + c] = v / L[(size_t)i * lda + i];
        }
        for (int i = N - 1; i >= 0; --i) {
            double v = B[(size_t)i * ldb + c];
            for (int l = i + 1; l < N; ++l) v -= L[(size_t)l * lda + i] * B[(size_t)l * ldb + c];
            B[(size_t)i * ldb + c] = v / L[(size_t)i * lda + i];
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kAdjThreads) adjoint_single_kernel(const AdjInst* __restrict__ insts) {
    const AdjInst I = insts[blockIdx.x];
    const int n = I.n, k = I.k, m = I.m, f64 = I.in_f64;
    const double kap = I.kappa, dexp = I.d;
    __shared__ double red[kAdjThreads / 32];
    __shared__ double sflag;
    __shared__ int nact;
    __shared__ int budget_s;
    const int tid = threadIdx.x;
    double* Ftx = I.vk;
    double* Ftu = I.vk + k;
    double* OFtx = I.vk + 2 * k;
    double* OFtu = I.vk + 3 * k;
    double* tv = I.vk + 4 * k;
    const int ldw = m + 2;    // W: k x (1 + active constraints)
    const int lds = m + 1;

    // ---- classification, curvature, l1 norm and F^T x ------------------------
    double l1 = 0;
    for (int i = tid; i < n; i += kAdjThreads) {
        const double x = ld(I.w, i, f64);
        const double z = x - ld(I.w0, i, f64);
        const double c1 = I.lam2 * ld(I.s, i, f64);
        const double c2 = I.lam3 * ld(I.q, i, f64);
        const double yd = ld(I.yD, i, f64);
        signed char c = 0;
        if (x == 0.0) c = 1;
        else if (fabs(yd) < c1) c = 2;
        double ih = 0;
        if (c == 0) {
            const double az = fabs(z);
            const double h = 2.0 * kap * ld(I.D, i, f64) +
                             (c2 > 0 && az > 0 ? c2 * dexp * (dexp - 1.0) * pow(az, dexp - 2.0) : 0.0);
            ih = 1.0 / h;
        }
        I.cls[i] = c;
        I.invh[i] = ih;
        l1 += fabs(x);
    }
    l1 = block_sum(l1, red);
    for (int j = tid; j < k; j += kAdjThreads) {
        double a = 0;
        for (int i = 0; i < n; ++i) a += ld(I.F, (size_t)i * k + j, f64) * ld(I.w, i, f64);
        Ftx[j] = a;
    }
    // active constraints: the budget (sum |x| = 1 up to rounding) and the
    // exposure rows with a nonzero multiplier (relative to the largest one)
    if (tid == 0) {
        double ymax = 0;
        for (int j = 0; j < m; ++j) ymax = fmax(ymax, fabs(ld(I.yA, j, f64)));
        int r = 0;
        // FP32 outputs carry their rounding into the l1 norm
        budget_s = l1 >= 1.0 - (f64 ? 1e-10 : 1e-6);
        if (budget_s) I.rows[r++] = -1;
        for (int j = 0; j < m; ++j)
            if (ymax > 0 && fabs(ld(I.yA, j, f64)) > 1e-12 * ymax) I.rows[r++] = j;
        nact = r;
        I.flags[0] = r;
    }
    __syncthreads();
    const int r = nact;
    auto erow = [&](int c, int i) -> double {   // entry i of constraint row c on the free block
        const int j = I.rows[c];
        if (j < 0) {
            const double x = ld(I.w, i, f64);
            return x > 0 ? 1.0 : (x < 0 ? -1.0 : 0.0);
        }
        return ld(I.A, (size_t)j * n + i, f64);
    };

    // ---- Gram blocks over the free assets ------------------------------------
    // M = F_S^T diag(1/h) F_S (+ (2 kappa Omega)^{-1}), W = F_S^T diag(1/h) [g, E^T],
    // Sc = E diag(1/h) E^T, vr = E diag(1/h) g
    for (int e = tid; e < k * k; e += kAdjThreads) {
        const int a = e / k, b = e % k;
        if (b > a) continue;
        double acc = 0;
        for (int i = 0; i < n; ++i) {
            const double ih = I.invh[i];
            if (ih != 0) acc += ld(I.F, (size_t)i * k + a, f64) * ld(I.F, (size_t)i * k + b, f64) * ih;
        }
        I.M[(size_t)a * k + b] = acc;
        I.M[(size_t)b * k + a] = acc;
    }
    for (int e = tid; e < k * (r + 1); e += kAdjThreads) {
        const int a = e / (r + 1), c = e % (r + 1);
        double acc = 0;
        for (int i = 0; i < n; ++i) {
            const double ih = I.invh[i];
            if (ih != 0) acc += ld(I.F, (size_t)i * k + a, f64) * ih * (c == 0 ? ld(I.gw, i, f64) : erow(c - 1, i));
        }
        I.W[(size_t)a * ldw + c] = acc;
    }
    for (int e = tid; e < r * (r + 1); e += kAdjThreads) {
        const int a = e / (r + 1), c = e % (r + 1);
        double acc = 0;
        for (int i = 0; i < n; ++i) {
            const double ih = I.invh[i];
            if (ih != 0) acc += erow(a, i) * ih * (c == 0 ? ld(I.gw, i, f64) : erow(c - 1, i));
        }
        if (c == 0) I.vr[a] = acc;
        else I.Sc[(size_t)a * lds + (c - 1)] = acc;
    }
    __syncthreads();
    // (2 kappa Omega)^{-1}
    if (I.omega_diag) {
        for (int j = tid; j < k; j += kAdjThreads) I.M[(size_t)j * k + j] += 1.0 / (2.0 * kap * ld(I.Omega, j, f64));
        __syncthreads();
    } else {
        // (2 kappa Omega)^{-1} column by column from the Cholesky factor of 2 kappa Omega
        for (int e = tid; e < k * k; e += kAdjThreads) I.Oi[e] = 2.0 * kap * ld(I.Omega, e, f64);
        __syncthreads();
        if (!cholesky(I.Oi, k, k, &sflag)) {
            if (tid == 0) { I.flags[1] = 1; if (I.status_out) *I.status_out = 1; }
            return;
        }
        for (int c = 0; c < k; ++c) {
            for (int j = tid; j < k; j += kAdjThreads) tv[j] = (j == c) ? 1.0 : 0.0;
            __syncthreads();
            chol_solve(I.Oi, k, k, tv, 1, 1);
            for (int j = tid; j < k; j += kAdjThreads) I.M[(size_t)j * k + c] += tv[j];
            __syncthreads();
        }
    }
    // ---- Y = M^{-1} W ------------------------------------------------------------
    if (!cholesky(I.M, k, k, &sflag)) {
        if (tid == 0) I.flags[1] = 1;
        return;
    }
    // Y = M^{-1} [W_g, W_e] in Oi's storage (k x (r + 1); Oi is no longer needed)
    double* Y = I.Oi;
    for (int e = tid; e < k * (r + 1); e += kAdjThreads) Y[e] = I.W[(size_t)(e / (r + 1)) * ldw + e % (r + 1)];
    __syncthreads();
    chol_solve(I.M, k, k, Y, r + 1, r + 1);
    // Schur complement Sc -= W_e^T Y_e, rhs vr -= W_e^T Y_g
    for (int e = tid; e < r * (r + 1); e += kAdjThreads) {
        const int a = e / (r + 1), c = e % (r + 1);
        double acc = 0;
        for (int j = 0; j < k; ++j) acc += I.W[(size_t)j * ldw + 1 + a] * Y[(size_t)j * (r + 1) + c];
        if (c == 0) I.vr[a] -= acc;
        else I.Sc[(size_t)a * lds + (c - 1)] -= acc;
    }
    __syncthreads();
    double* nu = I.vr + (m + 2);
    if (r > 0) {
        for (int a = tid; a < r; a += kAdjThreads) nu[a] = I.vr[a];
        __syncthreads();
        if (!cholesky(I.Sc, r, lds, &sflag)) {
            if (tid == 0) { I.flags[1] = 2; if (I.status_out) *I.status_out = 2; }
            return;
        }
        chol_solve(I.Sc, r, lds, nu, 1, 1);
    }
    // t = Y_g - Y_e nu
    for (int j = tid; j < k; j += kAdjThreads) {
        double v = Y[(size_t)j * (r + 1)];
        for (int a = 0; a < r; ++a) v -= Y[(size_t)j * (r + 1) + 1 + a] * nu[a];
        tv[j] = v;
    }
    __syncthreads();
    // ---- u on the free block ------------------------------------------------------
    for (int i = tid; i < n; i += kAdjThreads) {
        const double ih = I.invh[i];
        double uu = 0;
        if (ih != 0) {
            double v = ld(I.gw, i, f64);
            for (int a = 0; a < r; ++a) v -= nu[a] * erow(a, i);
            for (int j = 0; j < k; ++j) v -= ld(I.F, (size_t)i * k + j, f64) * tv[j];
            uu = v * ih;
        }
        I.u[i] = uu;
    }
    __syncthreads();
    for (int j = tid; j < k; j += kAdjThreads) {
        double a = 0;
        for (int i = 0; i < n; ++i) a += ld(I.F, (size_t)i * k + j, f64) * I.u[i];
        Ftu[j] = a;
    }
    __syncthreads();
    for (int j = tid; j < k; j += kAdjThreads) {
        double ax = 0, au = 0;
        if (I.omega_diag) {
            const double o = ld(I.Omega, j, f64);
            ax = o * Ftx[j];
            au = o * Ftu[j];
        } else {
            for (int l = 0; l < k; ++l) {
                const double o = ld(I.Omega, (size_t)j * k + l, f64);
                ax += o * Ftx[l];
                au += o * Ftu[l];
            }
        }
        OFtx[j] = ax;
        OFtu[j] = au;
    }
    __syncthreads();
    // ---- assembly ----------------------------------------------------------------------
    double nub = 0;
    int first_box = 0;
    if (budget_s) { nub = nu[0]; first_box = 1; }
    for (int i = tid; i < n; i += kAdjThreads) {
        const double x = ld(I.w, i, f64);
        const double w0 = ld(I.w0, i, f64);
        const double z = x - w0;
        const double uu = I.u[i];
        const signed char c = I.cls[i];
        const double sg = z > 0 ? 1.0 : (z < 0 ? -1.0 : 0.0);
        const double c2 = I.lam3 * ld(I.q, i, f64);
        const double az = fabs(z);
        st(I.dalpha, i, uu, f64);
        st(I.dD, i, -2.0 * kap * x * uu, f64);
        st(I.ds, i, -I.lam2 * sg * uu, f64);
        st(I.dq, i, c == 0 ? -I.lam3 * dexp * pow(az, dexp - 1.0) * sg * uu : 0.0, f64);
        double dw0 = 0;
        if (c == 0) {
            dw0 = (c2 > 0 && az > 0) ? c2 * dexp * (dexp - 1.0) * pow(az, dexp - 2.0) * uu : 0.0;
        } else if (c == 2 && w0 != 0.0) {
            double fo = 0;
            for (int j = 0; j < k; ++j) fo += ld(I.F, (size_t)i * k + j, f64) * OFtu[j];
            dw0 = ld(I.gw, i, f64) - 2.0 * kap * fo - nub * (w0 > 0 ? 1.0 : -1.0);
            for (int a = first_box; a < r; ++a) dw0 -= nu[a] * ld(I.A, (size_t)I.rows[a] * n + i, f64);
        }
        st(I.dw0, i, dw0, f64);
        if (I.dF) {
            for (int j = 0; j < k; ++j) st(I.dF, (size_t)i * k + j, -2.0 * kap * (uu * OFtx[j] + x * OFtu[j]), f64);
        }
    }
    if (tid == 0) { I.flags[1] = 0; if (I.status_out) *I.status_out = 0; }
}

inline size_t a256(size_t x) { return (x + 255) / 256 * 256; }

size_t adj_bytes(int n, int k, int m) {
    size_t b = 0;
    b += a256((size_t)n * 8);            // invh
    b += a256((size_t)n);                // cls
    b += a256((size_t)n * 8);            // u
    b += a256((size_t)(m + 1) * 4);      // rows
    b += a256((size_t)k * k * 8);        // M
    b += a256((size_t)k * std::max(k, m + 2) * 8);   // Oi (also the solved Y = M^{-1} W)
    b += a256((size_t)k * (m + 2) * 8);  // W
    b += a256((size_t)(m + 1) * (m + 1) * 8);  // Sc
    b += a256((size_t)4 * (m + 2) * 8);  // vr
    b += a256((size_t)6 * k * 8);        // vk
    b += a256(2 * 4);                    // flags
    return b;
}

}  // namespace
}  // namespace ff

namespace ff {
namespace {

bool valid_backward(const ff_problem* p, const void* w, const void* yA, const void* yD, const void* grad_w,
                    const ff_grads* out) {
    if (!p || p->T != 0 || !w || !yD || !grad_w || !out) return false;
    if (p->n < 1 || p->k < 1 || p->m < 0 || (p->m > 0 && (!yA || !p->A))) return false;
    if (p->dtype != FF_F64 && p->dtype != FF_F32) return false;
    if (!p->F || !p->Omega || !p->D || !p->alpha || !p->s || !p->q || !p->w0) return false;
    if (!(p->GMV > 0) || !(p->lambda1 > 0) || !(p->d > 1.0 && p->d <= 2.0)) return false;
    return true;
}

AdjInst carve_adj(const ff_problem* p, const void* w, const void* yA, const void* yD, const void* grad_w,
                  const ff_grads* out, unsigned char*& cur, int32_t* status_out) {
    AdjInst I;
    memset(&I, 0, sizeof(I));
    I.n = p->n; I.k = p->k; I.m = p->m; I.omega_diag = p->omega_diag ? 1 : 0; I.in_f64 = p->dtype == FF_F64;
    I.F = p->F; I.Omega = p->Omega; I.D = p->D; I.alpha = p->alpha; I.s = p->s; I.q = p->q; I.w0 = p->w0;
    I.A = p->A;
    I.w = w; I.yA = yA; I.yD = yD; I.gw = grad_w;
    I.dalpha = out->alpha; I.dF = out->F; I.dD = out->D; I.ds = out->s; I.dq = out->q; I.dw0 = out->w0;
    I.kappa = p->lambda1 * p->GMV; I.lam2 = p->lambda2; I.lam3 = p->lambda3; I.d = p->d;
    auto take = [&](size_t bytes) { unsigned char* r = cur; cur += a256(bytes); return (void*)r; };
    const int n = p->n, k = p->k, m = p->m;
    I.invh = (double*)take((size_t)n * 8);
    I.cls = (signed char*)take((size_t)n);
    I.u = (double*)take((size_t)n * 8);
    I.rows = (int*)take((size_t)(m + 1) * 4);
    I.M = (double*)take((size_t)k * k * 8);
    I.Oi = (double*)take((size_t)k * std::max(k, m + 2) * 8);
    I.W = (double*)take((size_t)k * (m + 2) * 8);
    I.Sc = (double*)take((size_t)(m + 1) * (m + 1) * 8);
    I.vr = (double*)take((size_t)4 * (m + 2) * 8);
    I.vk = (double*)take((size_t)6 * k * 8);
    I.flags = (int*)take(8);
    I.status_out = status_out;
    return I;
}

}  // namespace
}  // namespace ff

extern "C" {

int ff_backward_single(const ff_problem* p, const void* w, const void* yA, const void* yD, const void* grad_w,
                       const ff_grads* out, void* ws, size_t ws_bytes, int32_t* status_dev, void* stream);

size_t ff_backward_workspace_size(const ff_problem* p) {
    if (p && p->T >= 2) return ff_backward_multi_workspace_size(p, 1);
    if (!p || p->T != 0 || p->n < 1 || p->k < 1 || p->m < 0) return 0;
    return ff::a256(sizeof(ff::AdjInst)) + ff::adj_bytes(p->n, p->k, p->m);
}

size_t ff_backward_batch_workspace_size(const ff_problem* probs, int count) {
    if (!probs || count < 1) return 0;
    size_t b = ff::a256((size_t)count * sizeof(ff::AdjInst));
    for (int t = 0; t < count; ++t) {
        const ff_problem* p = &probs[t];
        if (p->T != 0 || p->n < 1 || p->k < 1 || p->m < 0) return 0;
        b += ff::adj_bytes(p->n, p->k, p->m);
    }
    return b;
}

int ff_backward_batch(const ff_problem* probs, int count, const void* const* w, const void* const* yA,
                      const void* const* yD, const void* const* grad_w, const ff_grads* out, void* ws,
                      size_t ws_bytes, int32_t* status_dev, void* stream) {
    if (!probs || count < 1 || count > 65535 || !w || !yD || !grad_w || !out) return FF_ERR_INVALID_ARG;
    for (int t = 0; t < count; ++t)
        if (!ff::valid_backward(&probs[t], w[t], yA ? yA[t] : nullptr, yD[t], grad_w[t], &out[t]))
            return FF_ERR_INVALID_ARG;
    const size_t need = ff_backward_batch_workspace_size(probs, count);
    if (!ws || ((uintptr_t)ws % 256) != 0 || ws_bytes < need) return FF_ERR_WORKSPACE;
    unsigned char* base = (unsigned char*)ws;
    unsigned char* cur = base + ff::a256((size_t)count * sizeof(ff::AdjInst));
    std::vector<ff::AdjInst> table(count);
    for (int t = 0; t < count; ++t)
        table[t] = ff::carve_adj(&probs[t], w[t], yA ? yA[t] : nullptr, yD[t], grad_w[t], &out[t], cur,
                                 status_dev ? status_dev + t : nullptr);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(base, table.data(), (size_t)count * sizeof(ff::AdjInst),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return FF_ERR_CUDA;
    ff::adjoint_single_kernel<<<count, ff::kAdjThreads, 0, st>>>((const ff::AdjInst*)base);
    e = cudaGetLastError();
    if (e != cudaSuccess) return FF_ERR_CUDA;
    return FF_OK;
}

int ff_backward(const ff_problem* p, const void* w, const void* yA, const void* yD, const void* grad_w,
                const ff_grads* out, void* ws, size_t ws_bytes, int32_t* status_dev, void* stream) {
    if (p && p->T >= 2) {
        const void* wv[1] = {w};
        const void* ya[1] = {yA};
        const void* yd[1] = {yD};
        const void* gv[1] = {grad_w};
        return ff_backward_multi_batch(p, 1, wv, ya, yd, gv, out, ws, ws_bytes, status_dev, stream);
    }
    return ff_backward_single(p, w, yA, yD, grad_w, out, ws, ws_bytes, status_dev, stream);
}

int ff_backward_single(const ff_problem* p, const void* w, const void* yA, const void* yD, const void* grad_w,
                       const ff_grads* out, void* ws, size_t ws_bytes, int32_t* status_dev, void* stream) {
    if (!ff::valid_backward(p, w, yA, yD, grad_w, out)) return FF_ERR_INVALID_ARG;
    const void* wv[1] = {w};
    const void* ya[1] = {yA};
    const void* yd[1] = {yD};
    const void* gv[1] = {grad_w};
    return ff_backward_batch(p, 1, wv, ya, yd, gv, out, ws, ws_bytes, status_dev, stream);
}

}  // extern "C"
