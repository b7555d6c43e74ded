// Risk-model estimation of Sec. 3.2 on the GPU, batched over estimation
// windows (one window per date; the paper uses the previous 504 business days):
//
//   Sigma_f = (F - 1 1^T F / T)^T (F - 1 1^T F / T) / (T - 1)
//   beta_i  = least squares of r_i ~ F beta_i over the days stock i has a return
//   D_ii    = sample variance of theta_{k,i} = r_{k,i} - beta_i^T f_k over those days
//
// A stock has returns from its first day in the window on (earlier days are
// NaN: a listing inside the window); a NaN after the first return makes it
// irregular.  Stocks with fewer than min_obs days, or irregular, are not
// estimated (beta = 0, D = NaN).
//
// One pass over R per window.  With first_i the stock's first day, its normal
// equations need G_i = sum_{k >= first_i} f_k f_k^T and g_i = sum_{k >= first_i} f_k,
// which depend on first_i only: risk_prep_kernel tabulates these suffix sums
// once per window in FP64 (products of FP32 inputs are exact in FP64), with
// Sigma_f.  risk_stream_kernel gives every stock one thread that streams its
// column: b = sum f_k r_k, s1 = sum r_k, s2 = sum r_k^2 are summed in FP32 over
// chunks of kChunk rows and each chunk sum is added into a double-float
// accumulator (an error-free two-sum), so the FP32 rounding is bounded by the
// chunk length; the 6x6 (p x p) solve and the variance are FP64.  The pass is
// bound by the HBM read of R (4 bytes per return).
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include "ff_internal.cuh"

namespace ff {
namespace {

constexpr int kRiskThreads = 256;
constexpr int kChunk = 8;          // rows summed in FP32 before a double-float fold
constexpr int kUnroll = 16;        // returns loaded ahead per thread
constexpr int kMaxP = 8;
constexpr int kMaxT = 4096;

__host__ __device__ inline int tri(int p) { return p * (p + 1) / 2; }

// per window: [T + 1][tri(p)] suffix Gram, [T + 1][p] suffix factor sums (FP64)
__host__ __device__ inline size_t window_doubles(int T, int p) { return (size_t)(T + 1) * (tri(p) + p); }

__global__ void risk_prep_kernel(const float* __restrict__ F, int T, int p, double* __restrict__ sigma_f,
                                 double* __restrict__ tables) {
    const int d = blockIdx.x;
    const float* f = F + (size_t)d * T * p;
    double* tab = tables + (size_t)d * window_doubles(T, p);
    const int np = tri(p);
    __shared__ double mean_s[kMaxP];
    // suffix sums: entry e < np is the Gram entry (a, b), a <= b; e >= np the sum of f_a
    for (int e = threadIdx.x; e < np + p; e += blockDim.x) {
        int a = 0, b = 0;
        if (e < np) {
            int r = e;
            while (r >= p - a) { r -= p - a; ++a; }
            b = a + r;
        } else {
            a = e - np;
        }
        double acc = 0.0;
        tab[(size_t)T * (np + p) + e] = 0.0;
        for (int k = T - 1; k >= 0; --k) {
            const double fa = (double)f[(size_t)k * p + a];
            acc += e < np ? fa * (double)f[(size_t)k * p + b] : fa;
            tab[(size_t)k * (np + p) + e] = acc;
        }
    }
    // factor covariance: mean-removed, divisor T - 1
    for (int a = threadIdx.x; a < p; a += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < T; ++k) s += (double)f[(size_t)k * p + a];
        mean_s[a] = s / (double)T;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const int a = e / p, b = e % p;
        double s = 0.0;
        for (int k = 0; k < T; ++k)
            s += ((double)f[(size_t)k * p + a] - mean_s[a]) * ((double)f[(size_t)k * p + b] - mean_s[b]);
        sigma_f[(size_t)d * p * p + e] = s / (double)(T - 1);
    }
}

// error-free fold of an FP32 chunk sum x into the pair (hi, lo)
__device__ __forceinline__ void fold(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

template <int P>
__global__ void __launch_bounds__(kRiskThreads)
risk_stream_kernel(const float* __restrict__ F, const float* __restrict__ R, int T, int n, int min_obs,
                   const double* __restrict__ tables, double* __restrict__ beta, double* __restrict__ D,
                   int32_t* __restrict__ nobs) {
    extern __shared__ float f_s[];   // [T][P] factor returns of this window
    const int d = blockIdx.y;
    const float* fw = F + (size_t)d * T * P;
    for (int e = threadIdx.x; e < T * P; e += blockDim.x) f_s[e] = fw[e];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* col = R + (size_t)d * T * n + i;
    float bh[P], bl[P], bc[P];
#pragma unroll
    for (int j = 0; j < P; ++j) { bh[j] = 0.f; bl[j] = 0.f; bc[j] = 0.f; }
    float s1h = 0.f, s1l = 0.f, s1c = 0.f, s2h = 0.f, s2l = 0.f, s2c = 0.f;
    int first = -1, inchunk = 0;
    bool regular = true;
    for (int k0 = 0; k0 < T; k0 += kUnroll) {
        float rv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) rv[u] = (k0 + u < T) ? __ldg(col + (size_t)(k0 + u) * n) : 0.f;
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int k = k0 + u;
            if (k >= T) break;
            const float r = rv[u];
            if (isnan(r)) {
                if (first >= 0) regular = false;
                continue;
            }
            if (first < 0) first = k;
            const float* fk = f_s + k * P;
#pragma unroll
            for (int j = 0; j < P; ++j) bc[j] = fmaf(fk[j], r, bc[j]);
            s1c += r;
            s2c = fmaf(r, r, s2c);
            if (++inchunk == kChunk) {
#pragma unroll
                for (int j = 0; j < P; ++j) { fold(bh[j], bl[j], bc[j]); bc[j] = 0.f; }
                fold(s1h, s1l, s1c);
                fold(s2h, s2l, s2c);
                s1c = 0.f;
                s2c = 0.f;
                inchunk = 0;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < P; ++j) fold(bh[j], bl[j], bc[j]);
    fold(s1h, s1l, s1c);
    fold(s2h, s2l, s2c);

    const int cnt = first < 0 ? 0 : T - first;
    double* bo = beta + ((size_t)d * n + i) * P;
    if (nobs) nobs[(size_t)d * n + i] = regular ? cnt : -1;
    if (!regular || cnt < min_obs || cnt < 2) {
#pragma unroll
        for (int j = 0; j < P; ++j) bo[j] = 0.0;
        D[(size_t)d * n + i] = NAN;
        return;
    }
    // normal equations G beta = b over the days k >= first (FP64 Cholesky)
    constexpr int NP = P * (P + 1) / 2;
    const double* tab = tables + (size_t)d * window_doubles(T, P) + (size_t)first * (NP + P);
    double Lm[P][P];
    {
        int e = 0;
        for (int a = 0; a < P; ++a)
            for (int b = a; b < P; ++b, ++e) { Lm[b][a] = tab[e]; Lm[a][b] = tab[e]; }
    }
    double b[P], g1[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
        b[j] = (double)bh[j] + (double)bl[j];
        g1[j] = tab[NP + j];
    }
    bool spd = true;
#pragma unroll
    for (int a = 0; a < P; ++a) {
        double s = Lm[a][a];
        for (int c = 0; c < a; ++c) s -= Lm[a][c] * Lm[a][c];
        if (!(s > 0.0)) { spd = false; s = 1.0; }
        const double l = sqrt(s);
        Lm[a][a] = l;
        for (int r = a + 1; r < P; ++r) {
            double t = Lm[r][a];
            for (int c = 0; c < a; ++c) t -= Lm[r][c] * Lm[a][c];
            Lm[r][a] = t / l;
        }
    }
    double y[P], x[P];
#pragma unroll
    for (int a = 0; a < P; ++a) {
        double t = b[a];
        for (int c = 0; c < a; ++c) t -= Lm[a][c] * y[c];
        y[a] = t / Lm[a][a];
    }
#pragma unroll
    for (int a = P - 1; a >= 0; --a) {
        double t = y[a];
        for (int c = a + 1; c < P; ++c) t -= Lm[c][a] * x[c];
        x[a] = t / Lm[a][a];
    }
    if (!spd) {
#pragma unroll
        for (int j = 0; j < P; ++j) bo[j] = 0.0;
        D[(size_t)d * n + i] = NAN;
        if (nobs) nobs[(size_t)d * n + i] = -2;
        return;
    }
    // residual moments: sum theta = s1 - beta^T g1, sum theta^2 = s2 - beta^T b (at the solution)
    double bt_b = 0.0, bt_g = 0.0;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        bo[j] = x[j];
        bt_b += x[j] * b[j];
        bt_g += x[j] * g1[j];
    }
    const double s1 = (double)s1h + (double)s1l;
    const double s2 = (double)s2h + (double)s2l;
    const double st = s1 - bt_g;
    const double sq = s2 - bt_b;
    D[(size_t)d * n + i] = (sq - st * st / (double)cnt) / (double)(cnt - 1);
}

template <int P>
cudaError_t launch_stream(const float* F, const float* R, int count, int T, int n, int min_obs,
                          const double* tables, double* beta, double* D, int32_t* nobs, cudaStream_t stream) {
    const size_t smem = (size_t)T * P * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(risk_stream_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((n + kRiskThreads - 1) / kRiskThreads), (unsigned)count);
    risk_stream_kernel<P><<<grid, kRiskThreads, smem, stream>>>(F, R, T, n, min_obs, tables, beta, D, nobs);
    return cudaGetLastError();
}

thread_local char g_risk_error[256] = "";

int risk_fail(cudaError_t e, const char* where) {
    snprintf(g_risk_error, sizeof(g_risk_error), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
    cudaGetLastError();
    return FF_ERR_CUDA;
}

}  // namespace
}  // namespace ff

extern "C" {

size_t ff_risk_workspace_size(int count, int T, int p) {
    if (count < 1 || count > 65535 || T < 2 || T > ff::kMaxT || p < 1 || p > ff::kMaxP) return 0;
    return (size_t)count * ff::window_doubles(T, p) * sizeof(double);
}

int ff_risk_estimate(int count, int T, int n, int p, const float* F, const float* R, int min_obs, double* beta,
                     double* sigma_f, double* D, int32_t* nobs, void* ws, size_t ws_bytes, void* stream) {
    const size_t need = ff_risk_workspace_size(count, T, p);
    if (need == 0 || n < 1 || min_obs < 2 || !F || !R || !beta || !sigma_f || !D) return FF_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws % 256) != 0 || ws_bytes < need) return FF_ERR_WORKSPACE;
    if ((long long)(n + ff::kRiskThreads - 1) / ff::kRiskThreads > 2147483647LL) return FF_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    double* tables = (double*)ws;
    ff::risk_prep_kernel<<<count, 64, 0, st>>>(F, T, p, sigma_f, tables);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return ff::risk_fail(e, "risk_prep_kernel launch");
    switch (p) {
        case 1: e = ff::launch_stream<1>(F, R, count, T, n, min_obs, tables, beta, D, nobs, st); break;
        case 2: e = ff::launch_stream<2>(F, R, count, T, n, min_obs, tables, beta, D, nobs, st); break;
        case 3: e = ff::launch_stream<3>(F, R, count, T, n, min_obs, tables, beta, D, nobs, st); break;
        case 4: e = ff::launch_stream<4>(F, R, count, T, n, min_obs, tables, beta, D, nobs, st); break;
        case 5: e = ff::launch_stream<5>(F, R, count, T, n, min_obs, tables, beta, D, nobs, st); break;
        case 6: e = ff::launch_stream<6>(F, R, count, T, n, min_obs, tables, beta, D, nobs, st); break;
        case 7: e = ff::launch_stream<7>(F, R, count, T, n, min_obs, tables, beta, D, nobs, st); break;
        default: e = ff::launch_stream<8>(F, R, count, T, n, min_obs, tables, beta, D, nobs, st); break;
    }
    if (e != cudaSuccess) return ff::risk_fail(e, "risk_stream_kernel launch");
    return FF_OK;
}

const char* ff_risk_last_error(void) { return ff::g_risk_error; }

}  // extern "C"
