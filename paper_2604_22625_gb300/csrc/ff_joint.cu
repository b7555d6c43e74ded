// Joint primal prox variant of the single-period solver (Sec. 2.1, Eqs. 1-3).
//
// The plain splitting of the solver kernel dualises the trading cost (its
// multiplier y_D) and projects onto the budget set.  This variant puts the
// cost and the budget set into one primal prox,
//     g(x) = phi(x - w0) + indicator{||x||_1 <= 1},
//     prox_{tau g}(v)_i = argmin_w 0.5 (w - v_i)^2 + tau phi_i(w - w0_i) + mu |w|,
// with mu >= 0 the budget's multiplier (scaled by tau): 0 when ||w(0)||_1 <= 1,
// else the root of ||w(mu)||_1 = 1, found by a safeguarded Newton iteration on
// mu.  Each coordinate problem has two kinks (at 0 and at w0_i) and is solved
// in closed form for d = 1.5 and d = 2 (a safeguarded Newton step otherwise).
// The only dual variable left is y_A of the exposure rows, so
//     x_bar = prox_{tau g}(x - tau (grad f(x) + A^T y_A)),
//     y_bar = p - sigma clip(p / sigma, L, U),  p = y_A + sigma A (2 x_bar - x),
// with the reflected Halpern scheme, the restarts and the relative KKT test of
// the plain solver (the trade multiplier of the KKT test is the cost's slope at
// x_bar - w0, or on the cost's kink the remainder of the prox's optimality
// condition, clipped to [-c1, c1]).  FP64 throughout; one CTA of 256
// threads per instance; the instance's arrays are converted to FP64 in the
// workspace (F transposed, factor-major, so that every matvec reads
// consecutive assets).
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "ff_internal.cuh"

namespace ff {
namespace {

constexpr int kJT = 256;           // threads of the CTA that solves one instance
constexpr int kJW = kJT / 32;      // its warps
constexpr int kJMaxK = 256;        // factors and exposure rows held in shared memory
constexpr int kJMaxM = 256;
constexpr int kMuRounds = 64;      // Newton / bisection rounds of the budget multiplier
constexpr int kThRounds = 64;      // rounds of the l1 threshold in the KKT test

struct JInst {
    int n, k, m, omega_diag, f64;
    double kappa, lam2, lam3, d, GMV;
    const void *F, *Omega, *D, *alpha, *s, *q, *w0, *A, *L, *U;
    void *w_out, *yA_out, *yD_out;
    ff_result* res;
    // workspace (FP64)
    double *FT;                    // k x n, factor-major
    double *Am;                    // m x n
    double *Om;                    // k x k, or k on the diagonal
    double *al, *Dd, *c1, *c2, *a; // n each: alpha, D, lambda2 s, lambda3 q, w0
    double *pd0;                   // n: phi_i'(-w0_i), the cost's slope at w = 0 (w0_i != 0)
    double *Lb, *Ub;               // m each
    double *x, *x0, *xb, *v, *qv, *ydb;   // n each
};

__device__ __forceinline__ double jld(const void* p, size_t i, int f64) {
    return f64 ? ((const double*)p)[i] : (double)((const float*)p)[i];
}
__device__ __forceinline__ void jst(void* p, size_t i, double v, int f64) {
    if (f64) ((double*)p)[i] = v;
    else ((float*)p)[i] = (float)v;
}
__device__ __forceinline__ double jsgn(double x) { return x > 0 ? 1.0 : (x < 0 ? -1.0 : 0.0); }

__device__ __forceinline__ double jwarp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums (or, for the entries flagged in maxmask, maxima) of NV values over the
// CTA, in a fixed order; every thread receives the totals.
template <int NV>
__device__ void jreduce(double (&v)[NV], double* red, unsigned maxmask = 0u) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < NV; ++e)
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_xor_sync(0xffffffffu, v[e], o);
            v[e] = ((maxmask >> e) & 1u) ? fmax(v[e], t) : v[e] + t;
        }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int e = 0; e < NV; ++e) red[warp * NV + e] = v[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < NV; ++e) {
        double t = red[e];
        for (int w = 1; w < kJW; ++w) t = ((maxmask >> e) & 1u) ? fmax(t, red[w * NV + e]) : t + red[w * NV + e];
        v[e] = t;
    }
    __syncthreads();
}

// out[j] = sum_i M[j n + i] vec[i] for j < rows (one warp per row, lanes over assets)
__device__ void jrows_apply(const double* M, int rows, int n, const double* vec, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = warp; j < rows; j += kJW) {
        const double* r = M + (size_t)j * n;
        double acc = 0;
        for (int i = lane; i < n; i += 32) acc += r[i] * vec[i];
        acc = jwarp_sum(acc);
        if (lane == 0) out[j] = acc;
    }
    __syncthreads();
}

// r >= 0 with r + gc d r^(d-1) = t for t > 0 (the impact part of the cost
// prox): closed form for d = 1.5 (rho = sqrt(r) solves rho^2 + 1.5 gc rho - t = 0,
// taken in its cancellation-free form) and d = 2; safeguarded Newton otherwise.
__device__ double impact_root(double t, double gc, double d, int dk) {
    if (!(t > 0.0)) return 0.0;
    if (!(gc > 0.0)) return t;
    if (dk == 1) {
        const double be = 1.5 * gc;
        const double rho = 2.0 * t / (be + sqrt(be * be + 4.0 * t));
        return rho * rho;
    }
    if (dk == 2) return t / (1.0 + 2.0 * gc);
    double lo = 0.0, hi = t, r = t;
    for (int it = 0; it < 100; ++it) {
        const double rp = pow(r, d - 1.0);
        const double h = r + gc * d * rp - t;
        if (h > 0) hi = r;
        else lo = r;
        const double dh = 1.0 + gc * d * (d - 1.0) * (r > 0 ? rp / r : 0.0);
        double rn = r - h / dh;
        if (!(rn > lo && rn < hi)) rn = 0.5 * (lo + hi);
        if (fabs(rn - r) <= 1e-16 * t) { r = rn; break; }
        r = rn;
    }
    return r;
}

// Coordinate problem of the joint prox:
//     w = argmin 0.5 (w - v)^2 + g (c1 |w - a| + c2 |w - a|^d) + mu |w|,
// and dwabs = d|w|/dmu (0 on a kink); cp0 = g phi'(-a), the cost's slope at
// w = 0 (a != 0).  The objective's derivative is monotone; its one-sided values
// at the kinks 0 and a decide whether the minimiser is a kink or which smooth
// piece holds it (signs s0 of w and s1 of w - a), where the optimality
// condition reduces to the impact root.
__device__ double joint_coord(double v, double a, double mu, double g, double c1, double c2, double cp0, double d,
                              int dk, double& dwabs) {
    const double gc1 = g * c1, gc2 = g * c2;
    dwabs = 0.0;
    const double lo_b = fmin(0.0, a), hi_b = fmax(0.0, a);
    // one-sided derivatives at a kink b (left Lb, right Rb)
    auto sides = [&](double b, double& Lb, double& Rb) {
        if (a == 0.0) {                       // both kinks at 0
            Lb = -v - gc1 - mu;
            Rb = -v + gc1 + mu;
        } else if (b == 0.0) {                // |w| kink, cost smooth at z = -a
            Lb = -v + cp0 - mu;
            Rb = -v + cp0 + mu;
        } else {                              // cost kink at w = a, |w| smooth
            const double base = (a - v) + mu * jsgn(a);
            Lb = base - gc1;
            Rb = base + gc1;
        }
    };
    double L1, R1;
    sides(lo_b, L1, R1);
    double s0, s1;
    if (L1 <= 0.0 && R1 >= 0.0) return lo_b;
    if (L1 > 0.0) {
        s0 = -1.0;
        s1 = -1.0;                            // below both kinks
    } else if (a == 0.0) {
        s0 = 1.0;
        s1 = 1.0;                             // above the single kink
    } else {
        double L2, R2;
        sides(hi_b, L2, R2);
        if (L2 <= 0.0 && R2 >= 0.0) return hi_b;
        if (L2 > 0.0) {                       // between the kinks
            s0 = a > 0 ? 1.0 : -1.0;
            s1 = a > 0 ? -1.0 : 1.0;
        } else {
            s0 = 1.0;
            s1 = 1.0;                         // above both kinks
        }
    }
    const double t = v - a - gc1 * s1 - mu * s0;
    const double r = impact_root(s1 * t, gc2, d, dk);
    const double w = a + s1 * r;
    if (r > 0.0 && w != 0.0) {
        double curv = 0.0;
        if (gc2 > 0.0) curv = gc2 * d * (d - 1.0) * (dk == 2 ? 1.0 : dk == 1 ? 1.0 / sqrt(r) : pow(r, d - 2.0));
        dwabs = -1.0 / (1.0 + curv);
    }
    return w;
}

__device__ __forceinline__ double cost_val(double z, double c1, double c2, double d) {
    const double az = fabs(z);
    return c1 * az + (c2 > 0 ? c2 * pow(az, d) : 0.0);
}

// phi*(y) for phi(z) = c1 |z| + c2 |z|^d
__device__ __forceinline__ double cost_conj_j(double y, double c1, double c2, double d) {
    const double e = fabs(y) - c1;
    if (!(e > 0)) return 0.0;
    if (!(c2 > 0)) return INFINITY;
    const double r = pow(e / (d * c2), 1.0 / (d - 1.0));
    return e * r * (1.0 - 1.0 / d);
}

__device__ __forceinline__ unsigned long long jclock() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void __launch_bounds__(kJT) joint_kernel(const JInst* __restrict__ insts, Params prm) {
    const JInst& I = insts[blockIdx.x];
    const int n = I.n, k = I.k, m = I.m, tid = threadIdx.x, f64 = I.f64;
    const double kap = I.kappa, dexp = I.d;
    const int dk = dexp == 1.5 ? 1 : (dexp == 2.0 ? 2 : 0);
    __shared__ double red[kJW * 16];
    __shared__ double uX[kJMaxK], u0[kJMaxK], uB[kJMaxK], wk[kJMaxK];
    __shared__ double yA[kJMaxM], yA0[kJMaxM], yAb[kJMaxM], ax[kJMaxM], ax0[kJMaxM], axb[kJMaxM];
    const unsigned long long t_start = jclock();
    unsigned long long ph[6] = {0, 0, 0, 0, 0, 0};
    unsigned long long t_mark = t_start;
    auto lap = [&](int q) {
        const unsigned long long t = jclock();
        ph[q] += t - t_mark;
        t_mark = t;
    };

    // ---- setup: FP64 copies, F transposed ----------------------------------
    for (size_t e = tid; e < (size_t)n * k; e += kJT) {
        const size_t i = e / k, j = e % k;
        I.FT[j * n + i] = jld(I.F, e, f64);
    }
    for (size_t e = tid; e < (size_t)n * m; e += kJT) I.Am[e] = jld(I.A, e, f64);
    for (int e = tid; e < (I.omega_diag ? k : k * k); e += kJT) I.Om[e] = jld(I.Omega, e, f64);
    for (int i = tid; i < n; i += kJT) {
        I.al[i] = jld(I.alpha, i, f64);
        I.Dd[i] = jld(I.D, i, f64);
        I.c1[i] = I.lam2 * jld(I.s, i, f64);
        I.c2[i] = I.lam3 * jld(I.q, i, f64);
        const double w = jld(I.w0, i, f64);
        I.a[i] = w;
        I.pd0[i] = w != 0.0 ? jsgn(-w) * (I.c1[i] + I.c2[i] * dexp * pow(fabs(w), dexp - 1.0)) : 0.0;
        I.x[i] = w;
        I.x0[i] = w;
    }
    for (int e = tid; e < m; e += kJT) {
        I.Lb[e] = jld(I.L, e, f64);
        I.Ub[e] = jld(I.U, e, f64);
        yA[e] = 0.0;
        yA0[e] = 0.0;
    }
    __syncthreads();
    // Omega u for a k-vector in shared memory (thread per factor)
    auto omega_times = [&](const double* u, double* out, double scale) {
        for (int j = tid; j < k; j += kJT) {
            double acc;
            if (I.omega_diag) acc = I.Om[j] * u[j];
            else {
                acc = 0;
                for (int l = 0; l < k; ++l) acc += I.Om[(size_t)j * k + l] * u[l];
            }
            out[j] = scale * acc;
        }
        __syncthreads();
    };

    // ---- Lipschitz constants: lambda_max(F Omega F^T + diag D), ||A||^2 ----
    double lamS = 0, lamA = 0;
    {
        double* p1 = I.v;     // power vectors live in v and qv until the iteration starts
        double* p2 = I.qv;
        for (int i = tid; i < n; i += kJT) {
            const double s = 1.0 + 0.25 * (double)((i * 2654435761u) % 1000u) / 1000.0;
            p1[i] = s;
            p2[i] = s;
        }
        __syncthreads();
        for (int it = 0; it < prm.power_iters; ++it) {
            jrows_apply(I.FT, k, n, p1, uB);
            omega_times(uB, wk, 1.0);
            if (m > 0) jrows_apply(I.Am, m, n, p2, axb);
            double nrm[2] = {0, 0};
            for (int i = tid; i < n; i += kJT) {
                double s1 = I.Dd[i] * p1[i];
                for (int j = 0; j < k; ++j) s1 += I.FT[(size_t)j * n + i] * wk[j];
                double s2 = 0;
                for (int j = 0; j < m; ++j) s2 += I.Am[(size_t)j * n + i] * axb[j];
                I.xb[i] = s1;
                I.ydb[i] = s2;
                nrm[0] += s1 * s1;
                nrm[1] += s2 * s2;
            }
            jreduce<2>(nrm, red);
            lamS = sqrt(nrm[0]);
            lamA = sqrt(nrm[1]);
            for (int i = tid; i < n; i += kJT) {
                p1[i] = lamS > 0 ? I.xb[i] / lamS : 0.0;
                p2[i] = lamA > 0 ? I.ydb[i] / lamA : 0.0;
            }
            __syncthreads();
        }
    }
    const double Lf = 2.0 * kap * lamS * 1.05;
    const double nA2 = m > 0 ? fmax(lamA * 1.05, 1e-300) : 1.0;
    const double tau = prm.step_fraction * 2.0 / Lf;
    // the whole dual budget 1/tau - beta L_f goes to the exposure rows
    const double sA = (1.0 / tau - prm.beta * Lf) / nA2;
    const double rho = prm.rho;

    // F^T x and A x of the start (w0); the anchors take the same values
    jrows_apply(I.FT, k, n, I.x, uX);
    if (m > 0) jrows_apply(I.Am, m, n, I.x, ax);
    for (int j = tid; j < k; j += kJT) u0[j] = uX[j];
    for (int j = tid; j < m; j += kJT) ax0[j] = ax[j];
    __syncthreads();
    lap(0);

    int status = FF_MAX_ITER, restarts = 0;
    long long it = 0, jh = 0, mu_rounds = 0;
    double mu_prev = 0.0;
    double r_restart = -1.0, r_prev = INFINITY, r_last = 0.0;
    double res_rel = INFINITY, res_p = 0, res_d = 0, res_g = 0, res_P = 0, res_D = 0, res_T = 0;
    for (it = 0; it < prm.max_iter; ++it) {
        // ---- gradient step: v = x - tau (grad f(x) + A^T y_A) --------------
        omega_times(uX, wk, 2.0 * kap);
        for (int i = tid; i < n; i += kJT) {
            double gr = -I.al[i] + 2.0 * kap * I.Dd[i] * I.x[i];
            for (int j = 0; j < k; ++j) gr += I.FT[(size_t)j * n + i] * wk[j];
            for (int j = 0; j < m; ++j) gr += I.Am[(size_t)j * n + i] * yA[j];
            I.v[i] = I.x[i] - tau * gr;
        }
        __syncthreads();
        lap(1);

        // ---- joint prox: the budget multiplier mu --------------------------
        double mu = 0.0;
        {
            auto S_at = [&](double mu_t, double& dS) {
                double sv[2] = {0.0, 0.0};
                for (int i = tid; i < n; i += kJT) {
                    double dw;
                    const double w = joint_coord(I.v[i], I.a[i], mu_t, tau, I.c1[i], I.c2[i], tau * I.pd0[i],
                                                 dexp, dk, dw);
                    sv[0] += fabs(w);
                    sv[1] += dw;
                }
                jreduce<2>(sv, red);
                ++mu_rounds;
                dS = sv[1];
                return sv[0];
            };
            // start at the previous iteration's mu; S(0) is evaluated only when
            // that point lies inside the budget (mu may then be 0)
            double lo = 0.0, hi = INFINITY, mt = mu_prev, dSt, St;
            bool search = true;
            if (mt > 0.0) {
                St = S_at(mt, dSt);
                if (St <= 1.0) {
                    double d0;
                    if (S_at(0.0, d0) <= 1.0) search = false;
                }
            } else {
                St = S_at(0.0, dSt);
                if (St <= 1.0) search = false;
            }
            if (search) {
                // bracket [lo, hi] with S(lo) > 1 >= S(hi); Newton steps, bisection
                // when a step leaves the bracket
                bool exact = false;
                for (int r = 0; r < kMuRounds; ++r) {
                    if (fabs(St - 1.0) <= 1e-15) { exact = true; break; }
                    if (St > 1.0) lo = mt;
                    else hi = mt;
                    if (isfinite(hi) && hi - lo <= 1e-16 * hi) break;
                    double mn = dSt < 0.0 ? mt + (St - 1.0) / (-dSt) : -1.0;
                    if (!(mn > lo && mn < hi))
                        mn = isfinite(hi) ? 0.5 * (lo + hi) : (lo > 0.0 ? 4.0 * lo : (St - 1.0) / (double)n);
                    mt = mn;
                    St = S_at(mt, dSt);
                }
                // a closed bracket ends on its budget side (S <= 1)
                mu = exact ? mt : (isfinite(hi) ? hi : mt);
            }
            mu_prev = mu;
        }
        lap(2);
        for (int i = tid; i < n; i += kJT) {
            double dw;
            I.xb[i] = joint_coord(I.v[i], I.a[i], mu, tau, I.c1[i], I.c2[i], tau * I.pd0[i], dexp, dk, dw);
        }
        __syncthreads();
        lap(3);

        // ---- F^T x_bar, A x_bar; dual step -----------------------------------
        jrows_apply(I.FT, k, n, I.xb, uB);
        if (m > 0) jrows_apply(I.Am, m, n, I.xb, axb);
        for (int j = tid; j < m; j += kJT) {
            const double p = yA[j] + sA * (2.0 * axb[j] - ax[j]);
            const double z = fmin(fmax(p / sA, I.Lb[j]), I.Ub[j]);
            yAb[j] = p - sA * z;
        }
        __syncthreads();
        lap(4);

        // ---- KKT test and restarts at (x_bar, y_bar) -----------------------
        const bool check = ((it + 1) % prm.check_every == 0) || (it + 1 == prm.max_iter);
        bool stop = false, do_restart = false;
        if (check) {
            // gradient at x_bar and the trade multiplier from the prox's optimality condition
            omega_times(uB, wk, 2.0 * kap);
            const double nu = mu / tau;
            double s[14] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int i = tid; i < n; i += kJT) {
                const double xb = I.xb[i], ai = I.a[i], c1 = I.c1[i], c2 = I.c2[i];
                double fw = 0;
                for (int j = 0; j < k; ++j) fw += I.FT[(size_t)j * n + i] * wk[j];
                const double gr = -I.al[i] + 2.0 * kap * I.Dd[i] * xb + fw;
                double aty = 0;
                for (int j = 0; j < m; ++j) aty += I.Am[(size_t)j * n + i] * yAb[j];
                // off the cost's kink the multiplier is phi'(x_bar - w0) (the one
                // subgradient there; exact, unlike the residual (v - x_bar) / tau - ...);
                // on the kink the optimality condition's remainder, clipped to [-c1, c1]
                double yd;
                if (xb != ai) {
                    const double z = xb - ai;
                    yd = jsgn(z) * (c1 + (c2 > 0 ? c2 * dexp * pow(fabs(z), dexp - 1.0) : 0.0));
                } else {
                    yd = fmin(fmax((I.v[i] - ai) / tau - nu * jsgn(ai), -c1), c1);
                }
                I.ydb[i] = yd;
                const double kty = aty + yd;
                I.qv[i] = xb - (gr + kty);
                const double dxi = I.x[i] - xb;
                s[0] += dxi * dxi;                                  // fixed-point residual (primal)
                s[1] += I.al[i] * xb;                               // alpha^T x
                s[2] += I.Dd[i] * xb * xb;                          // sum D x^2
                s[3] += cost_val(xb - ai, c1, c2, dexp);            // phi(x - w0)
                s[4] += fabs(I.al[i] * xb);                         // |alpha_i x_i|
                s[5] += gr * xb;                                    // <grad f, x>
                s[6] += yd * ai + cost_conj_j(yd, c1, c2, dexp);    // h_D*(y_D) = -<y, b> + phi*(y), b = -w0
                s[7] += xb * xb;
                s[8] += gr * gr;
                s[9] += kty * kty;
                s[10] = fmax(s[10], fabs(gr + kty));                // ||grad f + K^T y||_inf
                s[11] += fabs(I.qv[i]);
            }
            jreduce<14>(s, red, 1u << 10);
            // the projection of q onto the budget set: threshold by Newton's method
            double th = 0.0;
            if (s[11] > 1.0) {
                int nprev = -1;
                for (int r = 0; r < kThRounds; ++r) {
                    double tv[2] = {0.0, 0.0};
                    for (int i = tid; i < n; i += kJT) {
                        const double aq = fabs(I.qv[i]);
                        if (aq > th) { tv[0] += aq; tv[1] += 1.0; }
                    }
                    jreduce<2>(tv, red);
                    const int cnt = (int)tv[1];
                    const double tn = (tv[0] - 1.0) / (double)(cnt > 0 ? cnt : 1);
                    if (cnt == nprev || !(tn > th)) { th = fmax(tn, th); break; }
                    nprev = cnt;
                    th = tn;
                }
            }
            double pd[1] = {0.0};
            for (int i = tid; i < n; i += kJT) {
                const double qq = I.qv[i];
                const double pr = (s[11] > 1.0) ? jsgn(qq) * fmax(fabs(qq) - th, 0.0) : qq;
                const double e = I.xb[i] - pr;
                pd[0] += e * e;
            }
            jreduce<1>(pd, red);
            // exposure rows: residual, conjugate of the box, dual fixed-point part
            double pin = 0, nAx = 0, nCl = 0, hA = 0, rA = 0;
            for (int j = 0; j < m; ++j) {
                const double z = axb[j], cl = fmin(fmax(z, I.Lb[j]), I.Ub[j]);
                pin += (z - cl) * (z - cl);
                nAx += z * z;
                nCl += cl * cl;
                const double y = yAb[j];
                if (y > 0) hA += I.Ub[j] * y;
                if (y < 0) hA += I.Lb[j] * y;
                rA += (yA[j] - y) * (yA[j] - y);
            }
            double quad = 0;   // u^T (kappa Omega) u with u = F^T x_bar
            for (int j = 0; j < k; ++j) quad += uB[j] * wk[j];
            quad *= 0.5;
            const double fval = -s[1] + kap * s[2] + quad;
            const double Pobj = fval + s[3];
            const double Dobj = fval - s[5] - s[10] - hA - s[6];
            const double r_p = m > 0 ? sqrt(pin) / (sqrt(nAx) + sqrt(nCl) + 1e-30) : 0.0;
            const double r_d = sqrt(pd[0]) / (sqrt(s[7]) + sqrt(s[8]) + sqrt(s[9]) + 1e-30);
            const double r_g = fabs(Pobj - Dobj) / (fabs(Pobj) + fabs(Dobj) + 1e-30);
            const double rel = fmax(r_p, fmax(r_d, r_g));
            const double fpr = sqrt(s[0] / tau + rA / sA);
            res_rel = rel; res_p = r_p; res_d = r_d; res_g = r_g; res_P = Pobj; res_D = Dobj;
            res_T = s[4] + kap * s[2] + quad + s[3];
            r_last = fpr;
            const double tnow = (double)(jclock() - t_start);
            if (!(r_p == r_p) || !(r_d == r_d) || !(r_g == r_g) || !(fpr == fpr) || isinf(Pobj) || isinf(Dobj) ||
                !(Pobj == Pobj) || !(Dobj == Dobj)) {
                status = FF_NUMERICAL;
                res_rel = NAN;
                stop = true;
            } else if (rel <= prm.tol) {
                status = FF_CONVERGED;
                stop = true;
            } else if (tnow > prm.time_limit_ns) {
                status = FF_TIME_LIMIT;
                stop = true;
            } else {
                if (r_restart < 0) r_restart = fpr;
                do_restart = (fpr <= prm.beta_suff * r_restart) ||
                             (fpr <= prm.beta_nec * r_restart && fpr > r_prev) ||
                             (prm.beta_art > 0 && (double)jh >= prm.beta_art * (double)(it + 1));
                r_prev = fpr;
            }
            lap(5);
        }
        if (stop) break;

        // ---- reflected Halpern step ------------------------------------------
        const double lam = (double)(jh + 1) / (double)(jh + 2);
        for (int i = tid; i < n; i += kJT)
            I.x[i] = lam * ((1.0 + rho) * I.xb[i] - rho * I.x[i]) + (1.0 - lam) * I.x0[i];
        for (int j = tid; j < k; j += kJT) uX[j] = lam * ((1.0 + rho) * uB[j] - rho * uX[j]) + (1.0 - lam) * u0[j];
        for (int j = tid; j < m; j += kJT) {
            yA[j] = lam * ((1.0 + rho) * yAb[j] - rho * yA[j]) + (1.0 - lam) * yA0[j];
            ax[j] = lam * ((1.0 + rho) * axb[j] - rho * ax[j]) + (1.0 - lam) * ax0[j];
        }
        __syncthreads();
        ++jh;
        if (check) {
            // F^T x and A x recomputed from x at every check (the recursion above
            // carries them between checks)
            jrows_apply(I.FT, k, n, I.x, uX);
            if (m > 0) jrows_apply(I.Am, m, n, I.x, ax);
        }
        if (do_restart) {
            for (int i = tid; i < n; i += kJT) I.x0[i] = I.x[i];
            for (int j = tid; j < k; j += kJT) u0[j] = uX[j];
            for (int j = tid; j < m; j += kJT) { yA0[j] = yA[j]; ax0[j] = ax[j]; }
            __syncthreads();
            jh = 0;
            ++restarts;
            r_restart = r_last;
            r_prev = INFINITY;
        }
        lap(4);
    }

    // ---- outputs: x_bar, y_bar and the recovered trade multiplier of the last check
    for (int i = tid; i < n; i += kJT) {
        jst(I.w_out, i, I.xb[i], f64);
        if (I.yD_out) jst(I.yD_out, i, I.ydb[i], f64);
    }
    if (I.yA_out)
        for (int j = tid; j < m; j += kJT) jst(I.yA_out, j, yAb[j], f64);
    if (tid == 0) {
        ff_result rs;
        memset(&rs, 0, sizeof(rs));
        rs.status = status;
        rs.restarts = restarts;
        rs.iterations = (int64_t)(status == FF_MAX_ITER ? it : it + 1);
        rs.rel_kkt = res_rel;
        rs.r_primal = res_p;
        rs.r_dual = res_d;
        rs.r_gap = res_g;
        rs.primal_obj = res_P;
        rs.dual_obj = res_D;
        rs.paper_obj = -I.GMV * res_P;
        rs.fixed_point_res = r_last;
        rs.seconds = (double)(jclock() - t_start) * 1e-9;
        rs.lipschitz = Lf;
        rs.threshold_rounds = mu_rounds;
        for (int q = 0; q < 6; ++q) rs.phase_seconds[q] = (double)ph[q] * 1e-9;
        rs.term_scale = res_T;
        *I.res = rs;
    }
}

inline size_t j256(size_t x) { return (x + 255) / 256 * 256; }

size_t joint_inst_bytes(const ff_problem* p) {
    const size_t n = (size_t)p->n, k = (size_t)p->k, m = (size_t)p->m;
    return j256(k * n * 8) + j256(m * n * 8) + j256((p->omega_diag ? k : k * k) * 8) + 6 * j256(n * 8) +
           2 * j256(m * 8) + 6 * j256(n * 8);
}

}  // namespace

size_t joint_workspace_bytes(const ff_problem* probs, int count) {
    if (!probs || count < 1) return 0;
    size_t b = j256((size_t)count * sizeof(JInst));
    for (int t = 0; t < count; ++t) {
        const ff_problem* p = &probs[t];
        if (p->T != 0 || p->n < 1 || p->k < 1 || p->m < 0) return 0;
        b += joint_inst_bytes(p);
    }
    return b;
}

int joint_solve(const ff_problem* probs, int count, const Params& prm, void* ws, size_t ws_bytes, ff_result* res,
                void* const* w_out, void* const* yA_out, void* const* yD_out, cudaStream_t st, cudaError_t* cuda_err) {
    *cuda_err = cudaSuccess;
    for (int t = 0; t < count; ++t) {
        const ff_problem* p = &probs[t];
        if (p->T != 0) return FF_ERR_UNSUPPORTED;
        if (p->k > kJMaxK || p->m > kJMaxM) return FF_ERR_UNSUPPORTED;
        if (!w_out[t]) return FF_ERR_INVALID_ARG;
    }
    const size_t need = joint_workspace_bytes(probs, count);
    if (need == 0) return FF_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws % 256) != 0 || ws_bytes < need) return FF_ERR_WORKSPACE;
    unsigned char* base = (unsigned char*)ws;
    unsigned char* cur = base + j256((size_t)count * sizeof(JInst));
    auto take = [&](size_t bytes) { double* r = (double*)cur; cur += j256(bytes); return r; };
    std::vector<JInst> table(count);
    for (int t = 0; t < count; ++t) {
        const ff_problem* p = &probs[t];
        JInst& I = table[t];
        memset(&I, 0, sizeof(I));
        I.n = p->n; I.k = p->k; I.m = p->m; I.omega_diag = p->omega_diag ? 1 : 0;
        I.f64 = p->dtype == FF_F64;
        I.kappa = p->lambda1 * p->GMV; I.lam2 = p->lambda2; I.lam3 = p->lambda3; I.d = p->d; I.GMV = p->GMV;
        I.F = p->F; I.Omega = p->Omega; I.D = p->D; I.alpha = p->alpha; I.s = p->s; I.q = p->q; I.w0 = p->w0;
        I.A = p->A; I.L = p->L; I.U = p->U;
        I.w_out = w_out[t];
        I.yA_out = yA_out ? yA_out[t] : nullptr;
        I.yD_out = yD_out ? yD_out[t] : nullptr;
        I.res = res + t;
        const size_t n = (size_t)p->n, k = (size_t)p->k, m = (size_t)p->m;
        I.FT = take(k * n * 8);
        I.Am = take(m * n * 8);
        I.Om = take((p->omega_diag ? k : k * k) * 8);
        I.al = take(n * 8); I.Dd = take(n * 8); I.c1 = take(n * 8); I.c2 = take(n * 8); I.a = take(n * 8);
        I.pd0 = take(n * 8);
        I.Lb = take(m * 8); I.Ub = take(m * 8);
        I.x = take(n * 8); I.x0 = take(n * 8); I.xb = take(n * 8); I.v = take(n * 8); I.qv = take(n * 8);
        I.ydb = take(n * 8);
    }
    cudaError_t e = cudaMemcpyAsync(base, table.data(), (size_t)count * sizeof(JInst), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { *cuda_err = e; return FF_ERR_CUDA; }
    joint_kernel<<<count, kJT, 0, st>>>((const JInst*)base, prm);
    e = cudaGetLastError();
    if (e != cudaSuccess) { *cuda_err = e; return FF_ERR_CUDA; }
    return FF_OK;
}

}  // namespace ff
