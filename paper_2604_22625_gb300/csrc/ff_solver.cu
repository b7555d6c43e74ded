// Persistent "team" kernel: one thread-block cluster of G CTAs solves one
// portfolio instance at a time (single-period model, Sec. 2.1, or
// multi-period model, Sec. 2.2) and then takes the next instance of the batch.
//
// Method: restarted, reflected Halpern iteration of the Condat-Vu primal-dual
// splitting (the paper only states that its first-order method stops on a
// fixed-point residual, Sec. 4.1).  With K x = (A x_1..A x_P ; Delta x):
//   x_bar  = Proj_{||.||_1 <= 1}( x - tau (grad f(x) + K^T y) )        per period
//   y_bar  = prox_{sigma h*}( y + sigma K (2 x_bar - x) )
//            h_A = indicator[L, U] -> clip form; h_D = phi(. + b) -> Moreau with
//            the closed-form prox of c1 |z| + c2 |z|^d (d = 1.5, 2; Newton otherwise)
//   z+     = (j+1)/(j+2) ((1+rho) T(z) - rho z) + 1/(j+2) z_anchor
// grad f(x)_p = -alpha_p + 2 kappa (F Omega F^T (x_p - c) + D_p (x_p - c)).
//
// Work split inside a team: CTA g owns the assets [i0, i1).  Two passes over
// the panels per iteration:
//   expand (thread per asset, factor-major F^T and A):  F (Omega u), A^T y_A
//   reduce (thread per row, asset-major F and A^T):     A x_bar, F^T x_new, A x_new
// Sums over assets across the CTAs of the cluster go through distributed
// shared memory (each CTA adds one slice over all ranks in fixed order and
// writes it back to every rank), so every CTA holds bit-identical totals and
// takes identical control-flow decisions.  All waits are hardware cluster
// barriers; there is no spin loop.
#include <cooperative_groups.h>
#include <math.h>

#include "ff_internal.cuh"

namespace cg = cooperative_groups;

namespace ff {

// ---------------------------------------------------------------------------
// shared-memory layout (identical on host and device)
// ---------------------------------------------------------------------------
struct Layout {
    size_t vpart, vout;          // real, vlen each
    size_t spart, sout;          // double, slen each
    size_t wred;                 // double, kWarps * 32
    size_t stage;                // real, 4 * kPC * 32
    size_t yA, yAb, ax, ab;      // real, P*m each
    size_t u, ub, om;            // real, P*k each
    size_t Om;                   // real, k*k or k
    size_t cand, thprev, theta;  // double, P*kCand, P, P
    size_t lb, ub_;              // real, m each (exposure bounds)
    size_t total;
    int vlen, slen;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline Layout make_layout(int P, int k, int m, int omega_diag, size_t rs) {
    Layout L;
    L.vlen = P * (2 * m + 2 * k);
    if (L.vlen < 2) L.vlen = 2;
    int s1 = P * kCand * 2;
    int s2 = 4 * P + 32;
    L.slen = s1 > s2 ? s1 : s2;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 16); return r; };
    L.vpart = take((size_t)L.vlen * rs);
    L.vout = take((size_t)L.vlen * rs);
    L.spart = take((size_t)L.slen * 8);
    L.sout = take((size_t)L.slen * 8);
    L.wred = take((size_t)kWarps * 32 * 8);
    L.stage = take((size_t)4 * kPC * 32 * rs);
    L.yA = take((size_t)P * m * rs + 16);
    L.yAb = take((size_t)P * m * rs + 16);
    L.ax = take((size_t)P * m * rs + 16);
    L.ab = take((size_t)P * m * rs + 16);
    L.u = take((size_t)P * k * rs);
    L.ub = take((size_t)P * k * rs);
    L.om = take((size_t)P * k * rs);
    L.Om = take((size_t)(omega_diag ? k : k * k) * rs);
    L.cand = take((size_t)P * kCand * 8);
    L.thprev = take((size_t)P * 8);
    L.theta = take((size_t)P * 8);
    L.lb = take((size_t)m * rs + 16);
    L.ub_ = take((size_t)m * rs + 16);
    L.total = o;
    return L;
}

size_t solver_smem_bytes(int P, int k, int m, int omega_diag, size_t real_size) {
    return make_layout(P, k, m, omega_diag, real_size).total;
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float cvt(float a) { return a; }
__device__ __forceinline__ double cvt(double a) { return a; }
__device__ __forceinline__ float cvt(__nv_bfloat16 a) { return __bfloat162float(a); }

template <class real, class S>
__device__ __forceinline__ real ldp(const S* p) { return (real)cvt(__ldg(p)); }

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <class real>
__device__ __forceinline__ real warp_sum(real v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Scalar prox of gamma * (c1 |z| + c2 |z|^d) at t (Sec. 2.1 cost, one asset).
template <class real>
__device__ __forceinline__ real prox_cost(real t, real gamma, real c1, real c2, real d) {
    real a = fabs(t) - gamma * c1;
    if (!(a > (real)0)) return (real)0;
    real r;
    real gc = gamma * c2;
    if (gc <= (real)0) {
        r = a;
    } else if (d == (real)1.5) {
        // r + 1.5 gc sqrt(r) = a  ->  rho = sqrt(r) solves rho^2 + beta rho - a = 0
        real beta = (real)1.5 * gc;
        real rho = (real)2 * a / (beta + sqrt(beta * beta + (real)4 * a));
        r = rho * rho;
    } else if (d == (real)2) {
        r = a / ((real)1 + (real)2 * gc);
    } else {
        // safeguarded Newton on h(r) = r + gc d r^(d-1) - a over [0, a]
        real lo = 0, hi = a;
        r = a;
        for (int it = 0; it < 60; ++it) {
            real rp = pow(r, d - (real)1);
            real h = r + gc * d * rp - a;
            if (h > 0) hi = r; else lo = r;
            real dh = (real)1 + gc * d * (d - (real)1) * (r > 0 ? rp / r : (real)0);
            real rn = r - h / dh;
            if (!(rn > lo && rn < hi)) rn = (real)0.5 * (lo + hi);
            if (fabs(rn - r) <= (real)1e-15 * a) { r = rn; break; }
            r = rn;
        }
    }
    return t < 0 ? -r : r;
}

// phi*(y) for phi(z) = c1 |z| + c2 |z|^d  (Fenchel conjugate, per asset)
__device__ __forceinline__ double cost_conj(double y, double c1, double c2, double d) {
    double a = fabs(y) - c1;
    if (!(a > 0)) return 0.0;
    if (c2 <= 0) return INFINITY;
    double r = pow(a / (d * c2), 1.0 / (d - 1.0));
    return a * r * (1.0 - 1.0 / d);
}

// ---------------------------------------------------------------------------
// per-CTA context
// ---------------------------------------------------------------------------
template <class real, class S>
struct Ctx {
    Inst<real, S> I;
    int n, k, m, P, R, np;
    int i0, i1;
    int G, g;
    int tid, lane, warp;
    real* vpart;
    real* vout;
    double* spart;
    double* sout;
    double* wred;
    real* stage;
    real *yA, *yAb, *ax, *ab, *u, *ub, *om, *Om, *lb, *ubd;
    double *cand, *thprev, *theta;
};

// Sum (or max) of part[0..K) over the team; result in out[0..K) of every CTA.
template <class T, bool MAX>
__device__ void team_reduce(cg::cluster_group& cl, T* part, T* out, int K, int G, int g) {
    cl.sync();
    int per = (K + G - 1) / G;
    int lo = g * per;
    int hi = min(K, lo + per);
    for (int idx = lo + (int)threadIdx.x; idx < hi; idx += blockDim.x) {
        T s = MAX ? (T)-INFINITY : (T)0;
        for (int q = 0; q < G; ++q) {
            T v = cl.map_shared_rank(part, q)[idx];
            s = MAX ? (v > s ? v : s) : s + v;
        }
        for (int q = 0; q < G; ++q) cl.map_shared_rank(out, q)[idx] = s;
    }
    cl.sync();
}

// Block-wide sum of NV doubles held by every thread; thread 0..NV-1 of the block
// writes dst[i].  Ends with __syncthreads.
template <int NV>
__device__ void block_sum(double (&v)[NV], double* dst, double* wred, int lane, int warp) {
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) wred[warp * 32 + i] = v[i];
    }
    __syncthreads();
    if ((int)threadIdx.x < NV) {
        double s = 0;
        for (int w = 0; w < kWarps; ++w) s += wred[w * 32 + threadIdx.x];
        dst[threadIdx.x] = s;
    }
    __syncthreads();
}

template <int NV>
__device__ void block_max(double (&v)[NV], double* dst, double* wred, int lane, int warp) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] = fmax(v[i], __shfl_xor_sync(0xffffffffu, v[i], o));
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) wred[warp * 32 + i] = v[i];
    }
    __syncthreads();
    if ((int)threadIdx.x < NV) {
        double s = -INFINITY;
        for (int w = 0; w < kWarps; ++w) s = fmax(s, wred[w * 32 + threadIdx.x]);
        dst[threadIdx.x] = s;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// reduce pass: for every period p of the Pv-period vectors,
//   vpart[offA0 + p*m + j] = sum_i A_ji a0_pi     (and a1 into offA1)
//   vpart[offF0 + p*k + j] = sum_i F_ij (f0_pi - c_i) (and f1 into offF1)
// over the CTA's assets (thread per output row, asset-major panels).
// ---------------------------------------------------------------------------
template <class real, class S>
__device__ void reduce_pass(Ctx<real, S>& c, int Pv, const real* a0, const real* a1, const real* f0,
                            const real* f1, bool subcen, int offA0, int offA1, int offF0, int offF1) {
    const int m = c.m, k = c.k, np = c.np;
    const int rows = m + k;
    const S* Fam = c.I.Ft + (size_t)k * np;     // asset-major copy follows the factor-major one
    const S* Aam = c.I.At + (size_t)m * np;
    real* st = c.stage;                          // [4][kPC][32]
    for (int p0 = 0; p0 < Pv; p0 += kPC) {
        const int pc = min(kPC, Pv - p0);
        real acc[2][2][kPC];
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int t = 0; t < 2; ++t)
#pragma unroll
                for (int q = 0; q < kPC; ++q) acc[s][t][q] = 0;
        for (int ib = c.i0; ib < c.i1; ib += 32) {
            const int cnt = min(32, c.i1 - ib);
            // stage 4 vectors x pc periods x cnt assets
            for (int e = c.tid; e < 4 * kPC * 32; e += kThreads) {
                int vec = e / (kPC * 32);
                int q = (e / 32) % kPC;
                int ii = e % 32;
                real val = 0;
                if (q < pc && ii < cnt) {
                    int i = ib + ii;
                    size_t o = (size_t)(p0 + q) * np + i;
                    if (vec == 0) val = a0[o];
                    else if (vec == 1) val = a1 ? a1[o] : (real)0;
                    else if (vec == 2) val = f0[o] - (subcen ? c.I.cen[i] : (real)0);
                    else val = f1 ? f1[o] - (subcen ? c.I.cen[i] : (real)0) : (real)0;
                }
                st[e] = val;
            }
            __syncthreads();
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                int row = c.tid + s * kThreads;
                if (row < rows) {
                    bool isA = row < m;
                    int j = isA ? row : row - m;
                    const S* base = isA ? (Aam + (size_t)ib * m + j) : (Fam + (size_t)ib * k + j);
                    const int stride = isA ? m : k;
                    const real* sv0 = st + (isA ? 0 : 2) * kPC * 32;
                    const real* sv1 = st + (isA ? 1 : 3) * kPC * 32;
                    for (int ii = 0; ii < cnt; ++ii) {
                        real w = ldp<real, S>(base + (size_t)ii * stride);
#pragma unroll
                        for (int q = 0; q < kPC; ++q) {
                            acc[s][0][q] += w * sv0[q * 32 + ii];
                            acc[s][1][q] += w * sv1[q * 32 + ii];
                        }
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            int row = c.tid + s * kThreads;
            if (row < rows) {
                bool isA = row < m;
                int j = isA ? row : row - m;
#pragma unroll
                for (int q = 0; q < kPC; ++q) {
                    if (q < pc) {
                        int p = p0 + q;
                        if (isA) {
                            c.vpart[offA0 + p * m + j] = acc[s][0][q];
                            if (offA1 >= 0) c.vpart[offA1 + p * m + j] = acc[s][1][q];
                        } else {
                            c.vpart[offF0 + p * k + j] = acc[s][0][q];
                            if (offF1 >= 0) c.vpart[offF1 + p * k + j] = acc[s][1][q];
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// expand pass: for every local asset i and period p < Pv,
//   epi(i, p, (F wF_p)_i, (A^T wA_p)_i)     with wF (Pv x k), wA (Pv x m) in smem
// ---------------------------------------------------------------------------
template <class real, class S, class Epi>
__device__ void expand_pass(Ctx<real, S>& c, int Pv, const real* wF, const real* wA, Epi epi) {
    const int m = c.m, k = c.k, np = c.np;
    for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
        for (int p0 = 0; p0 < Pv; p0 += kPC) {
            real aF[kPC], aA[kPC];
#pragma unroll
            for (int q = 0; q < kPC; ++q) { aF[q] = 0; aA[q] = 0; }
            const int pc = min(kPC, Pv - p0);
            if (pc == kPC) {
                for (int j = 0; j < k; ++j) {
                    real f = ldp<real, S>(c.I.Ft + (size_t)j * np + i);
#pragma unroll
                    for (int q = 0; q < kPC; ++q) aF[q] += f * wF[(p0 + q) * k + j];
                }
                for (int j = 0; j < m; ++j) {
                    real a = ldp<real, S>(c.I.At + (size_t)j * np + i);
#pragma unroll
                    for (int q = 0; q < kPC; ++q) aA[q] += a * wA[(p0 + q) * m + j];
                }
            } else {
                for (int j = 0; j < k; ++j) {
                    real f = ldp<real, S>(c.I.Ft + (size_t)j * np + i);
#pragma unroll
                    for (int q = 0; q < kPC; ++q)
                        if (q < pc) aF[q] += f * wF[(p0 + q) * k + j];
                }
                for (int j = 0; j < m; ++j) {
                    real a = ldp<real, S>(c.I.At + (size_t)j * np + i);
#pragma unroll
                    for (int q = 0; q < kPC; ++q)
                        if (q < pc) aA[q] += a * wA[(p0 + q) * m + j];
                }
            }
#pragma unroll
            for (int q = 0; q < kPC; ++q)
                if (q < pc) epi(i, p0 + q, aF[q], aA[q]);
        }
    }
}

// om_p = Omega u_p for all periods (replicated in every CTA)
template <class real, class S>
__device__ void apply_omega(Ctx<real, S>& c, const real* uin, real* out, int Pv) {
    const int k = c.k;
    for (int e = c.tid; e < Pv * k; e += kThreads) {
        int p = e / k, j = e % k;
        real s;
        if (c.I.omega_diag) {
            s = c.Om[j] * uin[p * k + j];
        } else {
            s = 0;
            for (int l = 0; l < k; ++l) s += c.Om[j * k + l] * uin[p * k + l];
        }
        out[e] = s;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// l1-ball projection thresholds for every period of vector vv (P x np):
// theta_p >= 0 with sum_i max(|v_pi| - theta_p, 0) = 1, or 0 if ||v_p||_1 <= 1.
// Candidate-bracketing search: each round evaluates S(theta) = sum max(|v|-theta,0)
// and N(theta) = #{|v| > theta} at kCand candidates per period (FP64 sums);
// a Newton step from the largest candidate with S >= 1 is exact once no |v|
// lies between it and a candidate with S < 1 (equal counts).
// ---------------------------------------------------------------------------
template <class real, class S>
__device__ void l1_thresholds(cg::cluster_group& cl, Ctx<real, S>& c, const real* vv, double* th_out,
                              double* th_warm, bool* ok) {
    const int P = c.P, np = c.np;
    double* cand = c.cand;
    // round-0 candidates around the warm start
    for (int e = c.tid; e < P * kCand; e += kThreads) {
        int p = e / kCand, q = e % kCand;
        double w = th_warm[p];
        double val;
        if (q == 0 || !(w > 0)) val = (q == 0) ? 0.0 : w * 0.0 + (double)q * 1e-300;
        else {
            const double f[kCand] = {0.0, 0.9, 0.99, 0.999, 1.0, 1.001, 1.01, 1.1};
            val = w * f[q];
        }
        cand[e] = val;
    }
    // per-period done flags live in th_out sign: use a local array in smem (theta)
    __shared__ int done_s[64];
    for (int p = c.tid; p < 64; p += kThreads) done_s[p] = 0;
    __syncthreads();
    bool all_ok = true;
    for (int round = 0; round < kMaxRounds; ++round) {
        // local partial sums S, N per (period, candidate)
        for (int p = 0; p < P; ++p) {
            double acc[2 * kCand];
#pragma unroll
            for (int q = 0; q < 2 * kCand; ++q) acc[q] = 0;
            bool pd = (p < 64) ? done_s[p] : false;
            if (!pd) {
                double cq[kCand];
#pragma unroll
                for (int q = 0; q < kCand; ++q) cq[q] = cand[p * kCand + q];
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                    double a = fabs((double)vv[(size_t)p * np + i]);
#pragma unroll
                    for (int q = 0; q < kCand; ++q) {
                        double dlt = a - cq[q];
                        if (dlt > 0) { acc[q] += dlt; acc[kCand + q] += 1.0; }
                    }
                }
            }
            block_sum<2 * kCand>(acc, c.spart + p * 2 * kCand, c.wred, c.lane, c.warp);
        }
        team_reduce<double, false>(cl, c.spart, c.sout, P * 2 * kCand, c.G, c.g);
        // decisions (replicated, identical in every CTA)
        if (c.tid == 0) {
            for (int p = 0; p < P; ++p) {
                if (p < 64 && done_s[p]) continue;
                const double* Sv = c.sout + p * 2 * kCand;
                const double* Nv = Sv + kCand;
                double* cp = cand + p * kCand;
                if (round == 0 && Sv[0] <= 1.0) {   // inside the ball
                    th_out[p] = 0.0;
                    if (p < 64) done_s[p] = 1;
                    continue;
                }
                // largest candidate with S >= 1 (lower bracket) and smallest with S < 1
                int lo = -1, hi = -1;
                for (int q = 0; q < kCand; ++q) {
                    if (Sv[q] >= 1.0) { if (lo < 0 || cp[q] > cp[lo]) lo = q; }
                    else { if (hi < 0 || cp[q] < cp[hi]) hi = q; }
                }
                if (lo < 0) { lo = 0; }                 // cannot happen: candidate 0 keeps S >= 1
                double tl = cp[lo];
                double tn = tl + (Sv[lo] - 1.0) / fmax(Nv[lo], 1.0);
                bool exact = (hi >= 0 && Nv[hi] == Nv[lo]) || (Sv[lo] == 1.0);
                if (exact || round == kMaxRounds - 1) {
                    th_out[p] = tn;
                    if (!exact) all_ok = false;
                    if (p < 64) done_s[p] = 1;
                } else {
                    // next round: tn (a lower bound) and points towards the upper bracket
                    double th = (hi >= 0) ? cp[hi] : fmax(tn * 1.5, tn + 1e-12);
                    for (int q = 0; q < kCand; ++q)
                        cp[q] = tn + (th - tn) * (double)q / (double)kCand;
                }
            }
        }
        __syncthreads();
        int rem = 0;
        for (int p = 0; p < P && p < 64; ++p) rem += done_s[p] ? 0 : 1;
        if (rem == 0) break;
    }
    if (c.tid == 0) {
        for (int p = 0; p < P; ++p) th_warm[p] = th_out[p];
        *ok = all_ok;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <class real, class S>
__global__ void __launch_bounds__(kThreads, 1)
team_kernel(const Inst<real, S>* __restrict__ insts, int count, Params prm) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int G = (int)cl.num_blocks();
    const int g = (int)cl.block_rank();
    const int team = blockIdx.x / G;
    const int nteams = gridDim.x / G;

    for (int inst = team; inst < count; inst += nteams) {
        Ctx<real, S> c;
        c.I = insts[inst];
        c.n = c.I.n; c.k = c.I.k; c.m = c.I.m; c.P = c.I.P; c.R = c.I.R; c.np = c.I.np;
        c.G = G; c.g = g;
        c.tid = threadIdx.x; c.lane = threadIdx.x & 31; c.warp = threadIdx.x >> 5;
        c.i0 = (int)(((long long)c.n * g) / G);
        c.i1 = (int)(((long long)c.n * (g + 1)) / G);
        const int n = c.n, k = c.k, m = c.m, P = c.P, R = c.R, np = c.np;
        Layout Ly = make_layout(P, k, m, c.I.omega_diag, sizeof(real));
        c.vpart = (real*)(smem + Ly.vpart);
        c.vout = (real*)(smem + Ly.vout);
        c.spart = (double*)(smem + Ly.spart);
        c.sout = (double*)(smem + Ly.sout);
        c.wred = (double*)(smem + Ly.wred);
        c.stage = (real*)(smem + Ly.stage);
        c.yA = (real*)(smem + Ly.yA);
        c.yAb = (real*)(smem + Ly.yAb);
        c.ax = (real*)(smem + Ly.ax);
        c.ab = (real*)(smem + Ly.ab);
        c.u = (real*)(smem + Ly.u);
        c.ub = (real*)(smem + Ly.ub);
        c.om = (real*)(smem + Ly.om);
        c.Om = (real*)(smem + Ly.Om);
        c.cand = (double*)(smem + Ly.cand);
        c.thprev = (double*)(smem + Ly.thprev);
        c.theta = (double*)(smem + Ly.theta);
        c.lb = (real*)(smem + Ly.lb);
        c.ubd = (real*)(smem + Ly.ub_);
        const real kap = c.I.kappa;
        const real dexp = c.I.d;
        const unsigned long long t_start = globaltimer();

        // ---- prologue: replicated constants -------------------------------
        for (int e = c.tid; e < (c.I.omega_diag ? k : k * k); e += kThreads) c.Om[e] = c.I.Om[e];
        for (int e = c.tid; e < m; e += kThreads) { c.lb[e] = c.I.L[e]; c.ubd[e] = c.I.U[e]; }
        __syncthreads();

        // ---- Lipschitz constants by power iteration ----------------------
        // lambda_max(F Omega F^T + diag(Dmax)) and ||A||^2 = lambda_max(A A^T)
        double lamS = 0, lamA = 0;
        {
            real* v1 = c.I.pv1;
            real* v2 = c.I.pv2;
            for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                real s = (real)1 + (real)0.25 * (real)((i * 2654435761u) % 1000u) / (real)1000;
                v1[i] = s;
                v2[i] = s;
            }
            __syncthreads();
            for (int it = 0; it < prm.power_iters; ++it) {
                // F^T v1 (k) and A v2 (m)
                reduce_pass(c, 1, v2, (const real*)nullptr, v1, (const real*)nullptr, false, 0, -1, m, -1);
                team_reduce<real, false>(cl, c.vpart, c.vout, m + k, G, g);
                for (int e = c.tid; e < k; e += kThreads) c.u[e] = c.vout[m + e];
                for (int e = c.tid; e < m; e += kThreads) c.ax[e] = c.vout[e];
                __syncthreads();
                apply_omega(c, c.u, c.om, 1);
                // w1 = F om + Dmax v1,  w2 = A^T (A v2); norms
                double nrm[4] = {0, 0, 0, 0};
                expand_pass(c, 1, c.om, c.ax, [&](int i, int p, real aF, real aA) {
                    real w1 = aF + c.I.Dmax[i] * v1[i];
                    real w2 = aA;
                    nrm[0] += (double)w1 * w1;
                    nrm[1] += (double)w1 * v1[i];
                    nrm[2] += (double)w2 * w2;
                    nrm[3] += (double)w2 * v2[i];
                    c.I.xb[i] = w1;
                    c.I.xn[i] = w2;
                });
                block_sum<4>(nrm, c.spart, c.wred, c.lane, c.warp);
                team_reduce<double, false>(cl, c.spart, c.sout, 4, G, g);
                // v is a unit vector from the second step on, so ||Sigma v|| -> lambda_max
                double n1 = sqrt(c.sout[0]), n2 = sqrt(c.sout[2]);
                lamS = n1;
                lamA = n2;
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                    v1[i] = (real)(n1 > 0 ? c.I.xb[i] / n1 : 0.0);
                    v2[i] = (real)(n2 > 0 ? c.I.xn[i] / n2 : 0.0);
                }
                __syncthreads();
            }
        }
        const double Lf = 2.0 * (double)kap * lamS * 1.05;
        const double nA2 = (m > 0) ? fmax(lamA * 1.05, 1e-30) : 1.0;
        const double nD2 = c.I.multi ? 4.0 : 1.0;
        const double tau_d = prm.step_fraction * 2.0 / Lf;
        // sigma_A ||A||^2 + sigma_D ||Delta||^2 = 0.999 (1/tau - Lf/2), split evenly
        const double sig = 0.999 * (1.0 / tau_d - 0.5 * Lf) / ((m > 0) ? 2.0 : 1.0);
        const real tau = (real)tau_d;
        const real sA = (real)(sig / nA2);
        const real sD = (real)(sig / nD2);
        const real rho = (real)prm.rho;

        // ---- initial point: w0 (single) / straight line w0 -> w_T (multi) ----
        for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
            real w0 = c.I.w0[i];
            real wt = c.I.multi ? c.I.cen[i] : w0;
            for (int p = 0; p < P; ++p) {
                real x = c.I.multi ? w0 + (wt - w0) * (real)(p + 1) / (real)(P + 1) : w0;
                c.I.x[(size_t)p * np + i] = x;
                c.I.x0[(size_t)p * np + i] = x;
            }
            for (int r = 0; r < R; ++r) {
                c.I.yD[(size_t)r * np + i] = 0;
                c.I.yD0[(size_t)r * np + i] = 0;
            }
        }
        for (int e = c.tid; e < P * m; e += kThreads) c.yA[e] = 0;
        for (int p = c.tid; p < P; p += kThreads) c.thprev[p] = 0;
        __syncthreads();
        // u = F^T (x - c), ax = A x ; constant alpha_T^T w_T (multi)
        reduce_pass(c, P, c.I.x, (const real*)nullptr, c.I.x, (const real*)nullptr, true, 0, -1, 2 * P * m, -1);
        team_reduce<real, false>(cl, c.vpart, c.vout, 2 * P * m + P * k, G, g);
        for (int e = c.tid; e < P * m; e += kThreads) {
            c.ax[e] = c.vout[e];
            c.I.ax0[e] = c.vout[e];
            c.I.yA0[e] = 0;
        }
        for (int e = c.tid; e < P * k; e += kThreads) {
            c.u[e] = c.vout[2 * P * m + e];
            c.I.u0[e] = c.vout[2 * P * m + e];
        }
        double aTwT = 0;
        {
            double acc[1] = {0};
            if (c.I.multi)
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) acc[0] += (double)c.I.alphaT[i] * c.I.cen[i];
            block_sum<1>(acc, c.spart, c.wred, c.lane, c.warp);
            team_reduce<double, false>(cl, c.spart, c.sout, 1, G, g);
            aTwT = c.sout[0];
        }

        // ---- main loop ---------------------------------------------------------
        long long it = 0;
        int j = 0, restarts = 0;
        int status = FF_MAX_ITER;
        double r_restart = -1, r_prev = INFINITY, r_last = 0;
        double res_rel = INFINITY, res_p = 0, res_d = 0, res_g = 0, res_P = 0, res_D = 0;
        bool have_result = false;
        for (it = 0; it < prm.max_iter; ++it) {
            const bool check = (it % prm.check_every) == 0;
            const real cj = (real)(j + 1) / (real)(j + 2);
            const real oj = (real)1 - cj;
            // (1) om = Omega u
            apply_omega(c, c.u, c.om, P);
            // (2) expand: v = x - tau (grad f(x) + K^T y)
            {
                const real* x = c.I.x;
                const real* yD = c.I.yD;
                real* v = c.I.v;
                expand_pass(c, P, c.om, c.yA, [&](int i, int p, real aF, real aA) {
                    size_t o = (size_t)p * np + i;
                    real xv = x[o];
                    real g_ = -c.I.alpha[o] + (real)2 * kap * (aF + c.I.Dp[o] * (xv - c.I.cen[i]));
                    real kt = aA + yD[o] - ((p + 1 < R) ? yD[o + np] : (real)0);
                    v[o] = xv - tau * (g_ + kt);
                });
            }
            __syncthreads();
            // (3) thresholds
            bool thok;
            l1_thresholds(cl, c, c.I.v, c.theta, c.thprev, &thok);
            // (4) elementwise: x_bar, y_D bar, Halpern combination, residual parts
            double rloc[2] = {0, 0};
            {
                real* x = c.I.x;
                real* v = c.I.v;
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                    real xe_prev = 0;
                    real w0 = c.I.w0[i];
                    real wt = c.I.multi ? c.I.cen[i] : (real)0;
                    for (int r = 0; r < R; ++r) {
                        real xe = 0;
                        if (r < P) {
                            size_t o = (size_t)r * np + i;
                            real vv = v[o];
                            real th = (real)c.theta[r];
                            real av = fabs(vv) - th;
                            real xb = av > 0 ? (vv < 0 ? -av : av) : (real)0;
                            real xc = x[o];
                            c.I.xb[o] = xb;
                            xe = (real)2 * xb - xc;
                            c.I.xn[o] = cj * (((real)1 + rho) * xb - rho * xc) + oj * c.I.x0[o];
                            if (check) rloc[0] += (double)(xc - xb) * (xc - xb);
                        }
                        real dxe = xe - xe_prev;   // (Delta xe)_r, last multi row: -xe_{P-1}
                        xe_prev = xe;
                        real b = (r == 0 ? -w0 : (real)0) + ((c.I.multi && r == R - 1) ? wt : (real)0);
                        size_t orr = (size_t)r * np + i;
                        real yd = c.I.yD[orr];
                        real pD = yd + sD * dxe;
                        real t = pD / sD + b;
                        real pr = prox_cost<real>(t, (real)1 / sD, c.I.c1[orr], c.I.c2[orr], dexp);
                        real ydb = pD - sD * (pr - b);
                        c.I.yDb[orr] = ydb;
                        c.I.yDn[orr] = cj * (((real)1 + rho) * ydb - rho * yd) + oj * c.I.yD0[orr];
                        if (check) rloc[1] += (double)(yd - ydb) * (yd - ydb);
                    }
                }
            }
            __syncthreads();
            // (5) reduce: A x_bar, A x_new, F^T(x_new - c) [, F^T(x_bar - c)]
            reduce_pass(c, P, c.I.xb, c.I.xn, c.I.xn, check ? c.I.xb : (const real*)nullptr, true, 0, P * m,
                        2 * P * m, check ? 2 * P * m + P * k : -1);
            const int vlen = 2 * P * m + (check ? 2 : 1) * P * k;
            team_reduce<real, false>(cl, c.vpart, c.vout, vlen, G, g);
            // (6) replicated dual update of y_A, Halpern on (y_A, u, ax)
            double rA = 0;
            for (int e = c.tid; e < P * m; e += kThreads) {
                int jj = e % m;
                real abv = c.vout[e];
                real anv = c.vout[P * m + e];
                real ya = c.yA[e];
                real pA = ya + sA * ((real)2 * abv - c.ax[e]);
                real q = pA / sA;
                real cl_ = q > c.ubd[jj] ? c.ubd[jj] : (q < c.lb[jj] ? c.lb[jj] : q);
                real yab = pA - sA * cl_;
                c.yAb[e] = yab;
                c.ab[e] = abv;
                if (check) rA += (double)(ya - yab) * (ya - yab);
                c.yA[e] = cj * (((real)1 + rho) * yab - rho * ya) + oj * c.I.yA0[e];
                c.ax[e] = anv;
            }
            for (int e = c.tid; e < P * k; e += kThreads) {
                c.u[e] = c.vout[2 * P * m + e];
                if (check) c.ub[e] = c.vout[2 * P * m + P * k + e];
            }
            __syncthreads();
            // rotate iterate buffers: x <- x_new, y_D <- y_D new
            {
                real* t1 = c.I.x; c.I.x = c.I.xn; c.I.xn = t1;
                real* t2 = c.I.yD; c.I.yD = c.I.yDn; c.I.yDn = t2;
            }
            ++j;
            if (!check) continue;

            // ---- (7) check: fixed-point residual and relative KKT at T(z) --------
            // rA is per-thread over the replicated vector: every CTA computes it,
            // only rank 0 contributes so the team sum counts it once.
            double rr[3] = {rloc[0], rloc[1], (g == 0) ? rA : 0.0};
            block_sum<3>(rr, c.spart, c.wred, c.lane, c.warp);
            // KKT pieces at (x_bar, yA_bar, yD_bar)
            apply_omega(c, c.ub, c.om, P);
            double kloc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            {
                const real* xb = c.I.xb;
                const real* ydb = c.I.yDb;
                real* q = c.I.v;
                // the expand pass gives grad f(x_bar) and A^T yA_bar
                expand_pass(c, P, c.om, c.yAb, [&](int i, int p, real aF, real aA) {
                    size_t o = (size_t)p * np + i;
                    real xv = xb[o];
                    real dx = xv - c.I.cen[i];
                    real gf = -c.I.alpha[o] + (real)2 * kap * (aF + c.I.Dp[o] * dx);
                    real kt = aA + ydb[o] - ((p + 1 < R) ? ydb[o + np] : (real)0);
                    q[o] = xv - (gf + kt);
                    // f(x_bar) without the factor term: -alpha x + kappa D (x - c)^2
                    kloc[0] += (double)(-c.I.alpha[o]) * xv + (double)kap * c.I.Dp[o] * dx * dx;
                    kloc[1] += (double)gf * xv;         // <grad f, x>
                    kloc[2] += (double)xv * xv;
                    kloc[3] += (double)gf * gf;
                    kloc[4] += (double)kt * kt;
                });
                // trade costs: phi(Delta x_bar + b) and h_D*(yD_bar) = -<y, b> + sum phi*(y)
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                    real prevx = 0;
                    real w0 = c.I.w0[i];
                    real wt = c.I.multi ? c.I.cen[i] : (real)0;
                    for (int r = 0; r < R; ++r) {
                        real xv = (r < P) ? xb[(size_t)r * np + i] : (real)0;
                        real b = (r == 0 ? -w0 : (real)0) + ((c.I.multi && r == R - 1) ? wt : (real)0);
                        double z = (double)xv - (double)prevx + (double)b;
                        prevx = xv;
                        size_t orr = (size_t)r * np + i;
                        double c1 = c.I.c1[orr], c2 = c.I.c2[orr];
                        double az = fabs(z);
                        kloc[5] += c1 * az + c2 * pow(az, (double)dexp);
                        double y = ydb[orr];
                        kloc[6] += -y * b + cost_conj(y, c1, c2, (double)dexp);
                    }
                }
            }
            block_sum<8>(kloc, c.spart + 3, c.wred, c.lane, c.warp);
            // max_i |grad f + K^T y| per period  (g*(-grad f - K^T y) = sum_p max_i |.|)
            // and the timer of rank 0
            double tnow = (g == 0) ? (double)(globaltimer() - t_start) : 0.0;
            if (c.tid == 0) c.spart[11] = tnow;
            __syncthreads();
            team_reduce<double, false>(cl, c.spart, c.sout, 12, G, g);
            double sums[12];
            for (int e = 0; e < 12; ++e) sums[e] = c.sout[e];
            __syncthreads();
            // per-period max |x_bar - q| = |grad f + K^T y|
            for (int p = 0; p < P; ++p) {
                double mx[1] = {0};
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                    size_t o = (size_t)p * np + i;
                    mx[0] = fmax(mx[0], fabs((double)c.I.xb[o] - (double)c.I.v[o]));
                }
                block_max<1>(mx, c.spart + p, c.wred, c.lane, c.warp);
            }
            team_reduce<double, true>(cl, c.spart, c.sout, P, G, g);
            double gstar = 0;
            for (int p = 0; p < P; ++p) gstar += c.sout[p];
            __syncthreads();
            // projection of q = x_bar - (grad f + K^T y) for the stationarity residual
            double thq[64];
            {
                // thresholds for q, cold start (theta of this iteration is no longer needed)
                if (c.tid == 0) for (int p = 0; p < P; ++p) c.theta[p] = 0.0;
                __syncthreads();
                bool okq;
                l1_thresholds(cl, c, c.I.v, c.theta, c.theta, &okq);
                for (int p = 0; p < P && p < 64; ++p) thq[p] = c.theta[p];
            }
            double dr[1] = {0};
            for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                for (int p = 0; p < P; ++p) {
                    size_t o = (size_t)p * np + i;
                    double qv = c.I.v[o];
                    double aq = fabs(qv) - thq[p < 64 ? p : 63];
                    double pq = aq > 0 ? (qv < 0 ? -aq : aq) : 0.0;
                    double dd = (double)c.I.xb[o] - pq;
                    dr[0] += dd * dd;
                }
            }
            block_sum<1>(dr, c.spart, c.wred, c.lane, c.warp);
            team_reduce<double, false>(cl, c.spart, c.sout, 1, G, g);
            const double rd_num = sqrt(c.sout[0]);
            __syncthreads();
            // replicated pieces: factor part of f, h_A*(yA_bar), primal infeasibility
            double fF = 0, hA = 0, pin = 0, nAx = 0, nCl = 0;
            for (int e = 0; e < P * k; ++e) fF += (double)c.ub[e] * (double)c.om[e];
            for (int e = 0; e < P * m; ++e) {
                int jj = e % m;
                double y = c.yAb[e];
                if (y > 0) hA += y * (double)c.ubd[jj];
                else if (y < 0) hA += y * (double)c.lb[jj];
                double a = c.ab[e];
                double cla = fmin(fmax(a, (double)c.lb[jj]), (double)c.ubd[jj]);
                pin += (a - cla) * (a - cla);
                nAx += a * a;
                nCl += cla * cla;
            }
            const double fval = sums[3] + (double)kap * fF;
            const double Pobj = fval + sums[8];
            const double Dobj = fval - sums[4] - gstar - hA - sums[9];
            const double r_p = sqrt(pin) / (sqrt(nAx) + sqrt(nCl) + 1e-30);
            const double r_d = rd_num / (sqrt(sums[5]) + sqrt(sums[6]) + sqrt(sums[7]) + 1e-30);
            const double r_g = fabs(Pobj - Dobj) / (fabs(Pobj) + fabs(Dobj) + 1e-30);
            const double rel = fmax(r_p, fmax(r_d, r_g));
            const double fpr = sqrt(sums[0] / (double)tau + sums[1] / (double)sD + sums[2] / (double)sA);
            res_rel = rel; res_p = r_p; res_d = r_d; res_g = r_g; res_P = Pobj; res_D = Dobj;
            r_last = fpr;
            have_result = true;
            if (!(rel == rel) || !(fpr == fpr)) { status = FF_NUMERICAL; break; }
            if (rel <= prm.tol) { status = FF_CONVERGED; break; }
            if (sums[11] > prm.time_limit_ns) { status = FF_TIME_LIMIT; break; }
            // restart on the fixed-point residual (sufficient / necessary decay)
            if (r_restart < 0) r_restart = fpr;
            bool do_restart = (fpr <= prm.beta_suff * r_restart) || (fpr <= prm.beta_nec * r_restart && fpr > r_prev);
            r_prev = fpr;
            if (do_restart) {
                // z <- T(z): x = x0 = x_bar, yD = yD0 = yD_bar, yA = yA0 = yA_bar, u = u_bar, ax = a_bar
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                    for (int p = 0; p < P; ++p) {
                        size_t o = (size_t)p * np + i;
                        real xb = c.I.xb[o];
                        c.I.x[o] = xb;
                        c.I.x0[o] = xb;
                    }
                    for (int r = 0; r < R; ++r) {
                        size_t o = (size_t)r * np + i;
                        real y = c.I.yDb[o];
                        c.I.yD[o] = y;
                        c.I.yD0[o] = y;
                    }
                }
                for (int e = c.tid; e < P * m; e += kThreads) {
                    c.yA[e] = c.yAb[e];
                    c.I.yA0[e] = c.yAb[e];
                    c.ax[e] = c.ab[e];
                    c.I.ax0[e] = c.ab[e];
                }
                for (int e = c.tid; e < P * k; e += kThreads) {
                    c.u[e] = c.ub[e];
                    c.I.u0[e] = c.ub[e];
                }
                __syncthreads();
                j = 0;
                ++restarts;
                r_restart = fpr;
                r_prev = INFINITY;
            }
            (void)thok;
        }

        // ---- outputs: T(z) of the last check (x_bar, y_bar) -----------------
        __syncthreads();
        for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
            for (int p = 0; p < P; ++p) {
                double val = c.I.xb[(size_t)p * np + i];
                if (c.I.out_f64) ((double*)c.I.w_out)[(size_t)p * n + i] = val;
                else ((float*)c.I.w_out)[(size_t)p * n + i] = (float)val;
            }
            if (c.I.yD_out) {
                for (int r = 0; r < R; ++r) {
                    double val = c.I.yDb[(size_t)r * np + i];
                    if (c.I.out_f64) ((double*)c.I.yD_out)[(size_t)r * n + i] = val;
                    else ((float*)c.I.yD_out)[(size_t)r * n + i] = (float)val;
                }
            }
        }
        if (g == 0 && c.I.yA_out) {
            for (int e = c.tid; e < P * m; e += kThreads) {
                double val = c.yAb[e];
                if (c.I.out_f64) ((double*)c.I.yA_out)[e] = val;
                else ((float*)c.I.yA_out)[e] = (float)val;
            }
        }
        if (g == 0 && c.tid == 0) {
            ff_result rs;
            rs.status = have_result ? status : FF_MAX_ITER;
            rs.restarts = restarts;
            rs.iterations = (int64_t)it;
            rs.rel_kkt = res_rel;
            rs.r_primal = res_p;
            rs.r_dual = res_d;
            rs.r_gap = res_g;
            rs.primal_obj = res_P;
            rs.dual_obj = res_D;
            rs.paper_obj = c.I.GMV * (-res_P + aTwT);
            rs.fixed_point_res = r_last;
            rs.seconds = (double)(globaltimer() - t_start) * 1e-9;
            rs.lipschitz = Lf;
            *c.I.res = rs;
        }
        // the next instance reuses shared memory: all ranks must be done reading it
        cl.sync();
    }
}

template <class real, class S>
cudaError_t launch_solver(const Inst<real, S>* insts, int count, const Params& prm, int G, int nteams,
                          size_t smem, cudaStream_t stream) {
    auto kern = team_kernel<real, S>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (G > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(G * nteams), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, insts, count, prm);
}

template <class real, class S>
cudaError_t max_teams(int G, size_t smem, int* out) {
    auto kern = team_kernel<real, S>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (G > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(out, kern, &cfg);
}

template cudaError_t launch_solver<double, double>(const Inst<double, double>*, int, const Params&, int, int,
                                                   size_t, cudaStream_t);
template cudaError_t launch_solver<float, float>(const Inst<float, float>*, int, const Params&, int, int, size_t,
                                                 cudaStream_t);
template cudaError_t launch_solver<float, __nv_bfloat16>(const Inst<float, __nv_bfloat16>*, int, const Params&,
                                                         int, int, size_t, cudaStream_t);
template cudaError_t max_teams<double, double>(int, size_t, int*);
template cudaError_t max_teams<float, float>(int, size_t, int*);
template cudaError_t max_teams<float, __nv_bfloat16>(int, size_t, int*);

}  // namespace ff
