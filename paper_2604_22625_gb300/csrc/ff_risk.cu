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
// once per window as double-float pairs (exact products of the FP32 inputs,
// error-free sums in FP32 arithmetic: GB300's FP64 pipe is a small fraction of
// its FP32 pipe), with Sigma_f in FP64, and risk_ginv_kernel inverts G_j for
// every first day j in FP64.  risk_stream_kernel streams R once: per stock,
// b = sum f_k r_k, s1 = sum r_k, s2 = sum r_k^2 are summed in FP32
// over chunks of kChunk rows and each chunk sum is added into a double-float
// accumulator (an error-free two-sum), so the FP32 rounding is bounded by the
// chunk length; risk_finish_kernel applies the stock's inverse and forms the
// variance in FP64.  The pass over R is bound by its HBM read (4 bytes per
// return).
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include "ff_internal.cuh"

namespace ff {
namespace {

constexpr int kRiskThreads = 256;
constexpr int kChunk = 16;         // rows summed in FP32 before a double-float fold
constexpr int kBatch = 8;          // rows per register buffer of the streaming pass (two buffers)
constexpr int kMaxP = 8;
constexpr int kMaxT = 4096;

__host__ __device__ inline int tri(int p) { return p * (p + 1) / 2; }

// per window: [T + 1][tri(p)] suffix Gram, [T + 1][p] suffix factor sums
// (double-float pairs, 8 bytes each)
__host__ __device__ inline size_t window_doubles(int T, int p) { return (size_t)(T + 1) * (tri(p) + p); }

// (hi, lo) += a b exactly rounded to double-float: the product of two floats is
// p + e exactly (e from one FMA), added by an error-free two-sum
__device__ __forceinline__ void df_add_prod(float& hi, float& lo, float a, float b) {
    const float p = a * b;
    const float e = fmaf(a, b, -p);
    const float sm = hi + p;
    const float bb = sm - hi;
    lo += ((hi - (sm - bb)) + (p - bb)) + e;
    hi = sm;
}
__device__ __forceinline__ void df_add2(float& hi, float& lo, float bh, float bl) {
    const float sm = hi + bh;
    const float bb = sm - hi;
    lo += ((hi - (sm - bb)) + (bh - bb)) + bl;
    hi = sm;
}
__device__ __forceinline__ void df_norm(float& hi, float& lo) {
    const float sm = hi + lo;
    lo = lo - (sm - hi);
    hi = sm;
}

constexpr int kPrepSeg = 32;      // row segments of the suffix scan
constexpr int kCovPart = 16;      // partial sums per factor-covariance entry

// Per window: the suffix tables G_j = sum_{k >= j} f_k f_k^T (upper triangle) and
// g_j = sum_{k >= j} f_k as double-float pairs (FP32 arithmetic: each product of
// two FP32 inputs is exact as a pair, the sums are error-free two-sums, about
// 48 significant bits), and Sigma_f in FP64 from the mean-removed returns.
__global__ void __launch_bounds__(256) risk_prep_kernel(const float* __restrict__ F, int T, int p,
                                                        double* __restrict__ sigma_f, float2* __restrict__ tables,
                                                        int cen_smem) {
    extern __shared__ float fsh[];   // [T][p] factor returns of this window; then, with cen_smem,
                                     // [T][p] centred returns in FP64
    __shared__ float2 seg_tot[kPrepSeg][kMaxP * (kMaxP + 1) / 2 + kMaxP];
    __shared__ unsigned char ea_s[kMaxP * (kMaxP + 1) / 2], eb_s[kMaxP * (kMaxP + 1) / 2];
    __shared__ double mean_s[kMaxP];
    __shared__ double cov_part[kMaxP * kMaxP][kCovPart];
    const int d = blockIdx.x;
    const float* fg = F + (size_t)d * T * p;
    for (int e = threadIdx.x; e < T * p; e += blockDim.x) fsh[e] = fg[e];
    const int np = tri(p), ne = np + p;
    if (threadIdx.x == 0) {
        int e = 0;
        for (int a = 0; a < p; ++a)
            for (int b = a; b < p; ++b, ++e) { ea_s[e] = (unsigned char)a; eb_s[e] = (unsigned char)b; }
    }
    __syncthreads();
    const float* f = fsh;
    float2* tab = tables + (size_t)d * window_doubles(T, p);
    // entry e of row k: f_a f_b (e < np) or f_a (e >= np, as the product f_a * 1)
    auto factors = [&](int e, int k, float& x, float& y) {
        if (e < np) { x = f[(size_t)k * p + ea_s[e]]; y = f[(size_t)k * p + eb_s[e]]; }
        else { x = f[(size_t)k * p + (e - np)]; y = 1.0f; }
    };
    for (int w = threadIdx.x; w < ne * kPrepSeg; w += blockDim.x) {
        const int e = w % ne, sg = w / ne;
        const int k0 = (int)((long long)T * sg / kPrepSeg), k1 = (int)((long long)T * (sg + 1) / kPrepSeg);
        float hi = 0.f, lo = 0.f;
        for (int k = k0; k < k1; ++k) {
            float x, y;
            factors(e, k, x, y);
            df_add_prod(hi, lo, x, y);
        }
        df_norm(hi, lo);
        seg_tot[sg][e] = make_float2(hi, lo);
    }
    __syncthreads();
    for (int w = threadIdx.x; w < ne * kPrepSeg; w += blockDim.x) {
        const int e = w % ne, sg = w / ne;
        const int k0 = (int)((long long)T * sg / kPrepSeg), k1 = (int)((long long)T * (sg + 1) / kPrepSeg);
        float hi = 0.f, lo = 0.f;
        for (int q = kPrepSeg - 1; q > sg; --q) df_add2(hi, lo, seg_tot[q][e].x, seg_tot[q][e].y);   // later rows
        if (sg == kPrepSeg - 1) tab[(size_t)T * ne + e] = make_float2(0.f, 0.f);
        for (int k = k1 - 1; k >= k0; --k) {
            float x, y;
            factors(e, k, x, y);
            df_add_prod(hi, lo, x, y);
            df_norm(hi, lo);
            tab[(size_t)k * ne + e] = make_float2(hi, lo);
        }
    }
    // factor means from the segment totals, then the mean-removed covariance
    // (divisor T - 1) in FP64 with kCovPart partial sums per entry; the centred
    // returns are formed once in shared memory when they fit (cen_smem)
    if (threadIdx.x < p) {
        float hi = 0.f, lo = 0.f;
        for (int q = 0; q < kPrepSeg; ++q) df_add2(hi, lo, seg_tot[q][np + threadIdx.x].x, seg_tot[q][np + threadIdx.x].y);
        mean_s[threadIdx.x] = ((double)hi + (double)lo) / (double)T;
    }
    __syncthreads();
    double* cen = (double*)(fsh + ((size_t)T * p + 1) / 2 * 2);   // [T][p], 8-byte aligned after the floats
    if (cen_smem) {
        for (int e = threadIdx.x; e < T * p; e += blockDim.x) cen[e] = (double)f[e] - mean_s[e % p];
        __syncthreads();
    }
    for (int w = threadIdx.x; w < np * kCovPart; w += blockDim.x) {
        const int e = w % np, part = w / np;
        const int a = ea_s[e], b = eb_s[e];
        double sm = 0.0;
        if (cen_smem)
            for (int k = part; k < T; k += kCovPart) sm += cen[(size_t)k * p + a] * cen[(size_t)k * p + b];
        else
            for (int k = part; k < T; k += kCovPart)
                sm += ((double)f[(size_t)k * p + a] - mean_s[a]) * ((double)f[(size_t)k * p + b] - mean_s[b]);
        cov_part[a * p + b][part] = sm;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const int a = e / p, b = e % p;
        const int eu = a <= b ? e : b * p + a;   // the upper-triangle entry
        double sm = 0.0;
        for (int q = 0; q < kCovPart; ++q) sm += cov_part[eu][q];
        sigma_f[(size_t)d * p * p + e] = sm / (double)(T - 1);
    }
}

// Inverse of the Gram matrix G_j of every first day j < T of every window (one
// thread per (window, j)): FP64 Cholesky and P back-substitutions; the entry
// after the P x P inverse is 1 when G_j is positive definite, else 0.
template <int P>
__global__ void __launch_bounds__(64) risk_ginv_kernel(int T, const float2* __restrict__ tables,
                                                       double* __restrict__ ginv) {
    constexpr int NP = P * (P + 1) / 2;
    const int d = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= T) return;
    const float2* row = tables + (size_t)d * window_doubles(T, P) + (size_t)j * (NP + P);
    double Lm[P][P];
    {
        int e = 0;
#pragma unroll
        for (int a = 0; a < P; ++a)
#pragma unroll
            for (int b = a; b < P; ++b, ++e) {
                const float2 v = row[e];
                const double g = (double)v.x + (double)v.y;
                Lm[b][a] = g;
                Lm[a][b] = g;
            }
    }
    bool spd = true;
    double il[P];   // reciprocals of the factor's diagonal: one division per pivot
#pragma unroll
    for (int a = 0; a < P; ++a) {
        double sv = Lm[a][a];
#pragma unroll
        for (int c = 0; c < a; ++c) sv -= Lm[a][c] * Lm[a][c];
        if (!(sv > 0.0)) { spd = false; sv = 1.0; }
        const double l = sqrt(sv);
        il[a] = 1.0 / l;
        Lm[a][a] = l;
#pragma unroll
        for (int r = a + 1; r < P; ++r) {
            double t = Lm[r][a];
#pragma unroll
            for (int c = 0; c < a; ++c) t -= Lm[r][c] * Lm[a][c];
            Lm[r][a] = t * il[a];
        }
    }
    double* gi = ginv + ((size_t)d * T + j) * (P * P + 1);
#pragma unroll
    for (int col = 0; col < P; ++col) {
        double y[P], x[P];
#pragma unroll
        for (int a = 0; a < P; ++a) {
            double t = (a == col) ? 1.0 : 0.0;
#pragma unroll
            for (int c = 0; c < a; ++c) t -= Lm[a][c] * y[c];
            y[a] = t * il[a];
        }
#pragma unroll
        for (int a = P - 1; a >= 0; --a) {
            double t = y[a];
#pragma unroll
            for (int c = a + 1; c < P; ++c) t -= Lm[c][a] * x[c];
            x[a] = t * il[a];
        }
#pragma unroll
        for (int a = 0; a < P; ++a) gi[a * P + col] = x[a];
    }
    gi[P * P] = spd ? 1.0 : 0.0;
}

// error-free fold of an FP32 chunk sum x into the pair (hi, lo)
__device__ __forceinline__ void fold(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

// Streaming pass.  A thread holds two adjacent stocks (one 8-byte load per row
// when n is even) and walks every row of the window; the 8 warps of a block
// hold 512 consecutive stocks and walk the rows together, so each row is read
// as one contiguous 2 KB span per block (DRAM pages are read whole, not in
// scattered 256-byte pieces).  Two register buffers of kBatch rows keep the
// next rows' loads in flight while the current ones are summed.  Per stock:
// the double-float sums of f_k r_k (P), r_k, r_k^2, the first row with a
// return and the last row without one, written to the workspace for
// risk_finish_kernel.
constexpr int kStocks = 2 * 256;

template <int P, bool kVec>
__global__ void __launch_bounds__(256)
risk_stream_kernel(const float* __restrict__ F, const float* __restrict__ R, int T, int n,
                   double* __restrict__ sums, int* __restrict__ hist) {
    extern __shared__ float f_s[];   // [T][P] factor returns of this window
    constexpr int NS = P + 2;
    const int d = blockIdx.y;
    const float* fw = F + (size_t)d * T * P;
    for (int e = threadIdx.x; e < T * P; e += blockDim.x) f_s[e] = fw[e];
    __syncthreads();
    const int i0 = blockIdx.x * kStocks + 2 * threadIdx.x;
    if (i0 >= n) return;
    float hi[2][NS], lo[2][NS], ch[2][NS];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int j = 0; j < NS; ++j) { hi[q][j] = 0.f; lo[q][j] = 0.f; ch[q][j] = 0.f; }
    int first[2] = {1 << 30, 1 << 30}, lastnan[2] = {-1, -1}, inchunk = 0;
    const bool two = i0 + 1 < n;
    const float* col = R + (size_t)d * T * n + i0;
    // rows k0 .. k0 + kBatch - 1 of the stock pair (NaN past the window)
    auto load = [&](float2 (&rv)[kBatch], int k0) {
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int k = k0 + u;
            if (k < T) {
                const float* pk = col + (size_t)k * n;
                if constexpr (kVec) rv[u] = two ? __ldg((const float2*)pk) : make_float2(__ldg(pk), NAN);
                else rv[u] = make_float2(__ldg(pk), two ? __ldg(pk + 1) : NAN);
            } else {
                rv[u] = make_float2(NAN, NAN);
            }
        }
    };
    auto compute = [&](const float2 (&rv)[kBatch], int k0) {
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int k = k0 + u;
            if (k >= T) break;
            const float* fk = f_s + k * P;
            float fv[P];
#pragma unroll
            for (int j = 0; j < P; ++j) fv[j] = fk[j];
            const float r2[2] = {rv[u].x, rv[u].y};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const float r = r2[q];
                if (isnan(r)) { lastnan[q] = k; continue; }
                first[q] = min(first[q], k);
#pragma unroll
                for (int j = 0; j < P; ++j) ch[q][j] = fmaf(fv[j], r, ch[q][j]);
                ch[q][P] += r;
                ch[q][P + 1] = fmaf(r, r, ch[q][P + 1]);
            }
            // fold every kChunk rows (NaN rows count: a chunk holds at most kChunk terms)
            if (++inchunk == kChunk) {
#pragma unroll
                for (int q = 0; q < 2; ++q)
#pragma unroll
                    for (int j = 0; j < NS; ++j) { fold(hi[q][j], lo[q][j], ch[q][j]); ch[q][j] = 0.f; }
                inchunk = 0;
            }
        }
    };
    float2 ra[kBatch], rb[kBatch];
    load(ra, 0);
    for (int k0 = 0; k0 < T; k0 += 2 * kBatch) {
        load(rb, k0 + kBatch);
        compute(ra, k0);
        load(ra, k0 + 2 * kBatch);
        compute(rb, k0 + kBatch);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int ii = i0 + q;
        if (q == 1 && !two) break;
#pragma unroll
        for (int j = 0; j < NS; ++j) {
            fold(hi[q][j], lo[q][j], ch[q][j]);
            sums[((size_t)d * n + ii) * NS + j] = (double)hi[q][j] + (double)lo[q][j];
        }
        hist[2 * ((size_t)d * n + ii)] = first[q];
        hist[2 * ((size_t)d * n + ii) + 1] = lastnan[q];
    }
}

// beta and the residual variance from the moments: sum theta = s1 - beta^T g1,
// sum theta^2 = s2 - beta^T b (at the least-squares solution)
template <int P>
__device__ __forceinline__ void finish_moments(const double (&x)[P], const double (&b)[P], const double (&g1)[P],
                                               const double* s, int cnt, double* bo, double* Dout) {
    double bt_b = 0.0, bt_g = 0.0;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        bo[j] = x[j];
        bt_b += x[j] * b[j];
        bt_g += x[j] * g1[j];
    }
    const double st = s[P] - bt_g;
    const double sq = s[P + 1] - bt_b;
    *Dout = (sq - st * st / (double)cnt) / (double)(cnt - 1);
}

// One thread per stock: history rule, then beta = G_first^{-1} b from the
// window's precomputed inverse for the stock's first day, and the residual
// variance from the moments.
template <int P>
__global__ void risk_finish_kernel(int T, int n, int min_obs, const float2* __restrict__ tables,
                                   const double* __restrict__ ginv, const double* __restrict__ sums,
                                   const int* __restrict__ hist, double* __restrict__ beta, double* __restrict__ D,
                                   int32_t* __restrict__ nobs) {
    constexpr int NS = P + 2;
    const int d = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t si = (size_t)d * n + i;
    const int first = hist[2 * si], lastnan = hist[2 * si + 1];
    const bool any = first < T;
    const bool regular = !any || lastnan < first;
    const int cnt = any ? T - first : 0;
    double* bo = beta + si * P;
    if (nobs) nobs[si] = regular ? cnt : -1;
    const double* gi = ginv + ((size_t)d * T + (any ? first : 0)) * (P * P + 1);
    if (!regular || cnt < min_obs || cnt < 2 || gi[P * P] == 0.0) {
#pragma unroll
        for (int j = 0; j < P; ++j) bo[j] = 0.0;
        D[si] = NAN;
        if (nobs && regular && cnt >= min_obs && cnt >= 2) nobs[si] = -2;   // singular Gram matrix
        return;
    }
    constexpr int NP = P * (P + 1) / 2;
    const float2* tab = tables + (size_t)d * window_doubles(T, P) + (size_t)first * (NP + P);
    double b[P], g1[P], x[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
        b[j] = sums[si * NS + j];
        const float2 v = tab[NP + j];
        g1[j] = (double)v.x + (double)v.y;
    }
#pragma unroll
    for (int a = 0; a < P; ++a) {
        double t = 0.0;
#pragma unroll
        for (int c2 = 0; c2 < P; ++c2) t += gi[a * P + c2] * b[c2];
        x[a] = t;
    }
    finish_moments<P>(x, b, g1, sums + si * NS, cnt, bo, D + si);
}

template <int P>
cudaError_t launch_stream(const float* F, const float* R, int count, int T, int n, int min_obs,
                          const float2* tables, double* ginv, double* sums, int* hist, double* beta,
                          double* D, int32_t* nobs, cudaStream_t stream) {
    risk_ginv_kernel<P><<<dim3((unsigned)((T + 63) / 64), (unsigned)count), 64, 0, stream>>>(T, tables, ginv);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
    const size_t smem = (size_t)T * P * sizeof(float);
    // 8-byte row loads when every row of a thread's stock pair starts 8-byte aligned
    const bool vec = (n % 2 == 0) && ((uintptr_t)R % 8 == 0);
    auto kern = vec ? risk_stream_kernel<P, true> : risk_stream_kernel<P, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((n + kStocks - 1) / kStocks), (unsigned)count);
    kern<<<grid, 256, smem, stream>>>(F, R, T, n, sums, hist);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid2((unsigned)((n + 127) / 128), (unsigned)count);
    risk_finish_kernel<P><<<grid2, 128, 0, stream>>>(T, n, min_obs, tables, ginv, sums, hist, beta, D, nobs);
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

static size_t risk_tables_bytes(int count, int T, int p) {
    // suffix tables (double-float pairs), then the inverse Gram matrix of every
    // first day of every window (p^2 + 1 doubles each)
    return ((size_t)count * (ff::window_doubles(T, p) + (size_t)T * (p * p + 1)) * sizeof(double) + 255) / 256 * 256;
}

size_t ff_risk_workspace_size(int count, int T, int n, int p) {
    if (count < 1 || count > 65535 || T < 2 || T > ff::kMaxT || p < 1 || p > ff::kMaxP || n < 1) return 0;
    const size_t sums = ((size_t)count * n * (p + 2) * sizeof(double) + 255) / 256 * 256;
    const size_t hist = (size_t)count * n * 2 * sizeof(int);
    return risk_tables_bytes(count, T, p) + sums + hist;
}

int ff_risk_estimate(int count, int T, int n, int p, const float* F, const float* R, int min_obs, double* beta,
                     double* sigma_f, double* D, int32_t* nobs, void* ws, size_t ws_bytes, void* stream) {
    const size_t need = ff_risk_workspace_size(count, T, n, p);
    if (need == 0 || n < 1 || min_obs < 2 || !F || !R || !beta || !sigma_f || !D) return FF_ERR_INVALID_ARG;
    if (!ws || ((uintptr_t)ws % 256) != 0 || ws_bytes < need) return FF_ERR_WORKSPACE;
    if ((long long)(n + ff::kRiskThreads - 1) / ff::kRiskThreads > 2147483647LL) return FF_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    float2* tables = (float2*)ws;
    double* ginv = (double*)(tables + (size_t)count * ff::window_doubles(T, p));
    double* sums = (double*)((unsigned char*)ws + risk_tables_bytes(count, T, p));
    int* hist = (int*)((unsigned char*)sums + ((size_t)count * n * (p + 2) * sizeof(double) + 255) / 256 * 256);
    const size_t fsmem = (size_t)T * p * sizeof(float);
    // the centred returns in FP64 join the floats in shared memory when both fit in 160 KB
    const size_t csmem = ((size_t)T * p + 1) / 2 * 2 * sizeof(float) + (size_t)T * p * sizeof(double);
    const int cen_smem = csmem <= 160u * 1024u ? 1 : 0;
    const size_t psmem = cen_smem ? csmem : fsmem;
    cudaError_t e = cudaFuncSetAttribute(ff::risk_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    if (e != cudaSuccess) return ff::risk_fail(e, "risk_prep_kernel attribute");
    ff::risk_prep_kernel<<<count, 256, psmem, st>>>(F, T, p, sigma_f, tables, cen_smem);
    e = cudaGetLastError();
    if (e != cudaSuccess) return ff::risk_fail(e, "risk_prep_kernel launch");
    switch (p) {
        case 1: e = ff::launch_stream<1>(F, R, count, T, n, min_obs, tables, ginv, sums, hist, beta, D, nobs, st); break;
        case 2: e = ff::launch_stream<2>(F, R, count, T, n, min_obs, tables, ginv, sums, hist, beta, D, nobs, st); break;
        case 3: e = ff::launch_stream<3>(F, R, count, T, n, min_obs, tables, ginv, sums, hist, beta, D, nobs, st); break;
        case 4: e = ff::launch_stream<4>(F, R, count, T, n, min_obs, tables, ginv, sums, hist, beta, D, nobs, st); break;
        case 5: e = ff::launch_stream<5>(F, R, count, T, n, min_obs, tables, ginv, sums, hist, beta, D, nobs, st); break;
        case 6: e = ff::launch_stream<6>(F, R, count, T, n, min_obs, tables, ginv, sums, hist, beta, D, nobs, st); break;
        case 7: e = ff::launch_stream<7>(F, R, count, T, n, min_obs, tables, ginv, sums, hist, beta, D, nobs, st); break;
        default: e = ff::launch_stream<8>(F, R, count, T, n, min_obs, tables, ginv, sums, hist, beta, D, nobs, st); break;
    }
    if (e != cudaSuccess) return ff::risk_fail(e, "risk_stream_kernel launch");
    return FF_OK;
}

const char* ff_risk_last_error(void) { return ff::g_risk_error; }

}  // extern "C"
