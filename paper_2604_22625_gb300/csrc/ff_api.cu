// C ABI of the solver (declared in include/flashfolio.h): argument checks,
// workspace carving, panel repacking and the launch of the team kernel.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "ff_internal.cuh"

// Workspace of ff_solve_single_static: FF_STATIC_WORKSPACE_BYTES of device
// memory that every GPU which loads this library holds until the process
// exits.  Host code must not take its address directly (the host-side name is
// only a stand-in); it uses the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_ws[FF_STATIC_WORKSPACE_BYTES];

namespace ff {
namespace {

constexpr int kMaxStaticDevices = 64;

constexpr size_t kAlign = 256;

// Text of the last failed CUDA call on this host thread (ff_last_error).
thread_local char g_last_error[256] = "";

int cuda_fail(cudaError_t e, const char* where) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
    cudaGetLastError();   // clear a non-sticky launch error so the caller's stream stays usable
    return FF_ERR_CUDA;
}

inline size_t a256(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

inline size_t matvec_elem(int precision) { return precision == FF_PREC_F64 ? 8 : 4; }
inline size_t panel_elem(int precision) {
    return precision == FF_PREC_F64 ? 8 : (precision == FF_PREC_F32 ? 4 : 2);
}

struct Sizes {
    int n, k, m, P, R, np, multi;
    int omega_diag;
    Tiling tl;        // panel tiling; tl.CH == 0 when no tiling fits shared memory
};

inline Sizes sizes_of(const ff_problem& p, int precision) {
    Sizes s;
    s.n = p.n;
    s.k = p.k;
    s.m = p.m;
    s.multi = p.T >= 2;
    s.P = s.multi ? p.T - 1 : 1;
    s.R = s.multi ? p.T : 1;
    s.np = (p.n + 31) / 32 * 32;
    s.omega_diag = p.omega_diag ? 1 : 0;
    int vcap = 0, rep_glob = 0;
    const int CH = (s.P <= 64 && s.k + s.m <= 2 * kThreads)
                       ? choose_tile(s.P, s.n, s.k, s.m, s.omega_diag, matvec_elem(precision),
                                     panel_elem(precision), &vcap, &rep_glob)
                       : 0;
    s.tl = make_tiling(s.n, s.k, s.m, CH > 0 ? CH : 8, (int)panel_elem(precision));
    s.tl.CH = CH;
    s.tl.vcap = vcap;
    s.tl.rep_glob = rep_glob;
    return s;
}

inline size_t smem_of(const Sizes& s, int precision) {
    return solver_smem_bytes(s.P, s.k, s.m, s.omega_diag, matvec_elem(precision), s.tl.CH, s.tl.Rp,
                             panel_elem(precision), s.tl.vcap, s.tl.rep_glob);
}

inline size_t panel_bytes(const Sizes& s, int precision) {
    return (size_t)s.tl.ntile * s.tl.Rp * s.tl.CS * panel_elem(precision);
}

// bytes of workspace of one instance (excluding the Inst table); state is FP64
size_t inst_bytes(const Sizes& s, int omega_diag, int precision) {
    const size_t r = 8, pe = panel_elem(precision);
    size_t b = 0;
    b += a256(panel_bytes(s, precision));                   // panel tiles
    b += a256((size_t)(omega_diag ? s.k : s.k * s.k) * r);  // Omega
    b += 2 * a256((size_t)s.P * s.np * r);                  // alpha, D
    b += 4 * a256((size_t)s.np * r);                        // Dmax, w0, cen, alphaT
    b += 2 * a256((size_t)s.R * s.np * r);                  // c1, c2
    b += 2 * a256((size_t)s.m * r + 16);                    // L, U
    b += 5 * a256((size_t)s.P * s.np * r);                  // x, x0, xb, xn, v
    b += 4 * a256((size_t)s.R * s.np * r);                  // yD, yD0, yDb, yDn
    b += a256((size_t)s.P * s.m * r + 16);                  // yA0
    b += a256((size_t)s.R * s.np * 4);                      // yDf
    b += a256((size_t)s.np * 4);                            // cenf
    b += 2 * a256((size_t)s.np * 8);                        // w0f, cen2 (double-float pairs)
    b += 2 * a256((size_t)s.np * r);                        // power-iteration vectors
    if (s.tl.rep_glob) b += a256((size_t)kMaxCluster * rep_doubles(s.P, s.k, s.m) * r);   // replicated arrays
    return b;
}

// instance table + problem copies at the start of the workspace
constexpr size_t kQueueBytes = 256;   // per-group instance counters of the device queue
constexpr int kMaxGroups = 10;        // cluster sizes 1, 2, 4, 8, 16, single- or multi-period

template <class M, class S>
size_t table_bytes(int count) {
    return a256((size_t)count * sizeof(Inst<M, S>)) + a256((size_t)count * sizeof(ff_problem)) + kQueueBytes;
}

size_t table_bytes_of(int precision, int count) {
    return precision == FF_PREC_F64 ? table_bytes<double, double>(count)
                                    : (precision == FF_PREC_F32 ? table_bytes<float, float>(count)
                                                                : table_bytes<float, __nv_bfloat16>(count));
}

bool valid_problem(const ff_problem* p) {
    if (!p) return false;
    if (p->n < 1 || p->k < 1 || p->m < 0) return false;
    if (!(p->T == 0 || p->T >= 2)) return false;
    if (p->dtype != FF_F64 && p->dtype != FF_F32) return false;
    if (!p->F || !p->Omega || !p->D || !p->alpha || !p->s || !p->q || !p->w0) return false;
    if (p->m > 0 && (!p->A || !p->L || !p->U)) return false;
    if (p->T >= 2 && !p->wT) return false;
    if (!(p->GMV > 0) || !(p->lambda1 > 0) || !(p->lambda2 >= 0) || !(p->lambda3 >= 0)) return false;
    if (!(p->d > 1.0 && p->d <= 2.0)) return false;
    if (!isfinite(p->GMV) || !isfinite(p->lambda1) || !isfinite(p->lambda2) || !isfinite(p->lambda3))
        return false;
    return true;
}

bool supported(const Sizes& s, int omega_diag, int precision) {
    (void)omega_diag;
    (void)precision;
    if (s.P > 64) return false;              // per-period flags of the threshold search
    if (s.k + s.m > 2 * kThreads) return false;
    return s.tl.CH > 0;                      // a tiling whose layout fits shared memory
}

void fill_defaults(ff_options* o) {
    o->tol = 1e-6;
    o->max_iter = 400000;
    o->time_limit = 360.0;
    o->precision = FF_PREC_F32;
    o->check_every = 64;
    o->reflection = 1.0 / 3.0;
    o->restart_sufficient = 0.2;
    o->restart_necessary = 0.8;
    o->step_fraction = 0.4;
    o->beta = 0.75;
    o->reuse_workspace = 0;
    o->cta_work = 8192.0;
    o->restart_artificial = 0.36;
    o->cluster_size = 0;
    o->max_teams = 0;
    o->test_expire_first_wait = 0;
    o->stall_checks = 48;
    o->round_panels_bf16 = 0;
    o->warm_start = 0;
    o->panel_l2_keep = 1;
    o->primal_weight = 0;
}

bool valid_options(const ff_options& o) {
    if (!(o.tol > 0) || o.max_iter < 1 || !(o.time_limit > 0)) return false;
    if (o.precision < FF_PREC_F64 || o.precision > FF_PREC_BF16) return false;
    if (o.check_every < 1 || !(o.reflection >= 0 && o.reflection < 1)) return false;
    if (!(o.restart_sufficient > 0 && o.restart_sufficient < 1)) return false;
    if (!(o.restart_necessary > 0 && o.restart_necessary < 1)) return false;
    if (!(o.step_fraction > 0 && o.step_fraction < 1)) return false;
    // the dual steps need 1/tau - beta L_f > 0, i.e. 2 step_fraction beta < 1
    if (!(o.beta > 0.5) || !(2.0 * o.step_fraction * o.beta < 1.0)) return false;
    if (o.reflection > (2.0 * o.beta - 1.0) / (2.0 * o.beta) + 1e-12) return false;
    int g = o.cluster_size;
    if (!(g == 0 || g == 1 || g == 2 || g == 4 || g == 8 || g == 16)) return false;
    if (o.max_teams < 0) return false;
    if (o.reuse_workspace < 0 || o.reuse_workspace > 2) return false;
    if (!(o.cta_work >= 1.0)) return false;
    if (!(o.restart_artificial >= 0 && o.restart_artificial < 1)) return false;
    if (o.test_expire_first_wait != 0 && o.test_expire_first_wait != 1) return false;
    if (o.stall_checks < 0) return false;
    if (o.round_panels_bf16 != 0 && o.round_panels_bf16 != 1) return false;
    if (o.warm_start != 0 && o.warm_start != 1) return false;
    if (o.panel_l2_keep != 0 && o.panel_l2_keep != 1) return false;
    if (o.primal_weight != 0 && o.primal_weight != 1) return false;
    return true;
}

// ---------------------------------------------------------------------------
// repack kernel: caller arrays (paper layout, FP32/FP64) -> workspace layout
// ---------------------------------------------------------------------------
template <class S> __device__ __forceinline__ S to_s(double v);
template <> __device__ __forceinline__ double to_s<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_s<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_s<__nv_bfloat16>(double v) {
    return __float2bfloat16_rn((float)v);
}

template <class In, class M, class S>
__device__ void repack_one(const ff_problem& p, const Inst<M, S>& I, double lam2, double lam3, size_t tid,
                           size_t nth, int round_bf16) {
    const In* F = (const In*)p.F;
    const In* A = (const In*)p.A;
    const In* Om = (const In*)p.Omega;
    const In* D = (const In*)p.D;
    const In* al = (const In*)p.alpha;
    const In* s = (const In*)p.s;
    const In* q = (const In*)p.q;
    const In* w0 = (const In*)p.w0;
    const In* wT = (const In*)p.wT;
    const In* L = (const In*)p.L;
    const In* U = (const In*)p.U;
    const int n = I.n, k = I.k, m = I.m, P = I.P, R = I.R, np = I.np;
    // panel tiles: PE[t][r][ii] for asset i = t CH + ii (ii < CH; CS - CH pads)
    // and panel row r (F rows 0..k-1, A rows kp..kp+m-1, zero padding elsewhere)
    S* PE = (S*)I.PE;
    const int CH = I.CH, CS = I.CS, Rp = I.Rp, kp = I.kp;
    const size_t total = (size_t)I.ntile * Rp * CS;
    for (size_t e = tid; e < total; e += nth) {
        const int ii = (int)(e % CS);
        const int r = (int)((e / CS) % Rp);
        const int t = (int)(e / ((size_t)CS * Rp));
        const int i = t * CH + ii;
        double v = 0.0;
        if (ii < CH && i < n) {
            if (r < k) v = (double)F[(size_t)i * k + r];
            else if (r >= kp && r < kp + m) v = (double)A[(size_t)(r - kp) * n + i];
        }
        if (round_bf16) v = (double)__bfloat162float(__float2bfloat16_rn((float)v));
        PE[e] = to_s<S>(v);
    }
    const int nOm = I.omega_diag ? k : k * k;
    for (size_t e = tid; e < (size_t)nOm; e += nth) ((double*)I.Om)[e] = (double)Om[e];
    for (size_t e = tid; e < (size_t)m; e += nth) {
        ((double*)I.L)[e] = (double)L[e];
        ((double*)I.U)[e] = (double)U[e];
    }
    for (size_t e = tid; e < (size_t)np; e += nth) {
        int i = (int)e;
        bool in = i < n;
        double dmax = 0;
        for (int pp = 0; pp < P; ++pp) {
            double dv = in ? (double)D[(size_t)pp * n + i] : 0.0;
            double av = in ? (double)al[(size_t)pp * n + i] : 0.0;
            ((M*)I.Dp)[(size_t)pp * np + i] = (M)dv;
            ((M*)I.alpha)[(size_t)pp * np + i] = (M)av;
            dmax = fmax(dmax, dv);
        }
        ((double*)I.Dmax)[i] = (double)dmax;
        for (int r = 0; r < R; ++r) {
            ((M*)I.c1)[(size_t)r * np + i] = (M)(in ? lam2 * (double)s[(size_t)r * n + i] : 0.0);
            ((M*)I.c2)[(size_t)r * np + i] = (M)(in ? lam3 * (double)q[(size_t)r * n + i] : 0.0);
        }
        const double w0v = in ? (double)w0[i] : 0.0;
        const double cv = (in && I.multi) ? (double)wT[i] : 0.0;
        ((double*)I.w0)[i] = w0v;
        ((double*)I.cen)[i] = cv;
        ((float*)I.cenf)[i] = (float)cv;
        const float w0h = (float)w0v, ch = (float)cv;
        ((float2*)I.w0f)[i] = make_float2(w0h, (float)(w0v - (double)w0h));
        ((float2*)I.cen2)[i] = make_float2(ch, (float)(cv - (double)ch));
        if (I.multi) ((double*)I.alphaT)[i] = (double)(in ? (double)al[(size_t)P * n + i] : 0.0);
    }
}

// One launch repacks every instance of the batch: blockIdx.y selects the
// table slot, the blocks along x stride over that instance's elements.
template <class M, class S>
__global__ void repack_batch_kernel(const ff_problem* __restrict__ probs, const Inst<M, S>* __restrict__ insts,
                                    int round_bf16) {
    const ff_problem p = probs[blockIdx.y];
    const Inst<M, S> I = insts[blockIdx.y];
    const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const size_t nth = (size_t)gridDim.x * blockDim.x;
    if (p.dtype == FF_F64)
        repack_one<double, M, S>(p, I, p.lambda2, p.lambda3, tid, nth, round_bf16);
    else
        repack_one<float, M, S>(p, I, p.lambda2, p.lambda3, tid, nth, round_bf16);
}

template <class M, class S>
Inst<M, S> carve(const ff_problem& p, const Sizes& s, unsigned char*& cur, void* w_out, void* yA_out,
                 void* yD_out, ff_result* res) {
    Inst<M, S> I;
    memset(&I, 0, sizeof(I));
    I.n = s.n; I.k = s.k; I.m = s.m; I.P = s.P; I.R = s.R; I.multi = s.multi; I.np = s.np;
    I.omega_diag = p.omega_diag ? 1 : 0;
    auto take = [&](size_t bytes) { unsigned char* r = cur; cur += a256(bytes); return (void*)r; };
    const size_t r = sizeof(double);
    I.CH = s.tl.CH; I.CS = s.tl.CS; I.kp = s.tl.kp; I.mp = s.tl.mp; I.Rp = s.tl.Rp; I.ntile = s.tl.ntile;
    I.vcap = s.tl.vcap;
    const size_t pb = (size_t)s.tl.ntile * s.tl.Rp * s.tl.CS * sizeof(S);
    I.PE = (const S*)take(pb);
    I.Om = (const double*)take((size_t)(I.omega_diag ? s.k : s.k * s.k) * r);
    I.alpha = (const M*)take((size_t)s.P * s.np * r);
    I.Dp = (const M*)take((size_t)s.P * s.np * r);
    I.Dmax = (const double*)take((size_t)s.np * r);
    I.w0 = (const double*)take((size_t)s.np * r);
    I.cen = (const double*)take((size_t)s.np * r);
    I.alphaT = (const double*)take((size_t)s.np * r);
    I.c1 = (const M*)take((size_t)s.R * s.np * r);
    I.c2 = (const M*)take((size_t)s.R * s.np * r);
    I.L = (const double*)take((size_t)s.m * r + 16);
    I.U = (const double*)take((size_t)s.m * r + 16);
    I.x = (double*)take((size_t)s.P * s.np * r);
    I.x0 = (double*)take((size_t)s.P * s.np * r);
    I.xb = (double*)take((size_t)s.P * s.np * r);
    I.xn = (double*)take((size_t)s.P * s.np * r);
    I.v = (double*)take((size_t)s.P * s.np * r);
    I.yD = (double*)take((size_t)s.R * s.np * r);
    I.yD0 = (double*)take((size_t)s.R * s.np * r);
    I.yDb = (double*)take((size_t)s.R * s.np * r);
    I.yDn = (double*)take((size_t)s.R * s.np * r);
    I.yA0 = (double*)take((size_t)s.P * s.m * r + 16);
    I.yDf = (float*)take((size_t)s.R * s.np * 4);
    I.cenf = (const float*)take((size_t)s.np * 4);
    I.w0f = (const float2*)take((size_t)s.np * 8);
    I.cen2 = (const float2*)take((size_t)s.np * 8);
    I.pv1 = (double*)take((size_t)s.np * r);
    I.pv2 = (double*)take((size_t)s.np * r);
    I.rep_glob = s.tl.rep_glob;
    I.rep = s.tl.rep_glob ? (double*)take((size_t)kMaxCluster * rep_doubles(s.P, s.k, s.m) * r) : nullptr;
    I.kappa = p.lambda1 * p.GMV;
    I.d = p.d;
    I.GMV = p.GMV;
    I.w_out = w_out;
    I.yA_out = yA_out;
    I.yD_out = yD_out;
    I.out_f64 = p.dtype == FF_F64;
    I.res = res;
    return I;
}

// Cluster size of every instance of a batch.  Each instance starts with the
// smallest power of two G that keeps its asset-periods per CTA at or below
// cta_work; while the whole batch would occupy fewer than half the SMs, the
// instance with the most work per CTA is split further (down to 384
// asset-periods per CTA), so that a small batch, or one instance, still
// spreads over the GPU.
void choose_clusters(const std::vector<Sizes>& sz, double cta_work, int sms, std::vector<int>& G) {
    const int count = (int)sz.size();
    G.assign(count, 1);
    long long total = 0;
    for (int t = 0; t < count; ++t) {
        const double ap = (double)sz[t].n * sz[t].P;
        while (G[t] < 16 && ap > (double)G[t] * cta_work) G[t] *= 2;
        total += G[t];
    }
    while (total < sms / 2) {
        int best = -1;
        double bw = 0;
        for (int t = 0; t < count; ++t) {
            const double per = (double)sz[t].n * sz[t].P / G[t];
            if (G[t] < 16 && per > 2.0 * 384 && per > bw) { bw = per; best = t; }
        }
        if (best < 0) break;
        total += G[best];
        G[best] *= 2;
    }
}

// Side streams (one per cluster-size group; side[0] has the highest
// priority) and fork/join events, created once per device under
// g_streams_mu, which also serialises the fork/join enqueue.
struct DeviceStreams {
    bool ready = false;
    cudaStream_t side[kMaxGroups];
    cudaEvent_t fork;
    cudaEvent_t join[kMaxGroups];
};
std::mutex g_streams_mu;
DeviceStreams g_streams[kMaxStaticDevices];

int device_streams(DeviceStreams** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxStaticDevices) return FF_ERR_UNSUPPORTED;
    DeviceStreams& d = g_streams[dev];
    if (!d.ready) {
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e != cudaSuccess) return cuda_fail(e, "stream priority range");
        for (int i = 0; i < kMaxGroups; ++i) {
            const int prio = std::max(greatest, least - (kMaxGroups - 1 - i));
            e = cudaStreamCreateWithPriority(&d.side[i], cudaStreamNonBlocking, prio);
            if (e != cudaSuccess) return cuda_fail(e, "side stream creation");
            e = cudaEventCreateWithFlags(&d.join[i], cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(e, "event creation");
        }
        e = cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "event creation");
        d.ready = true;
    }
    *out = &d;
    return FF_OK;
}

Params make_params(const ff_options& o) {
    Params prm;
    prm.tol = o.tol;
    prm.max_iter = o.max_iter;
    prm.time_limit_ns = o.time_limit * 1e9;
    prm.check_every = o.check_every;
    prm.rho = o.reflection;
    prm.beta_suff = o.restart_sufficient;
    prm.beta_nec = o.restart_necessary;
    prm.beta_art = o.restart_artificial;
    prm.step_fraction = o.step_fraction;
    prm.beta = o.beta;
    prm.power_iters = 60;
    prm.expire_first_wait = o.test_expire_first_wait;
    prm.stall_checks = o.stall_checks;
    prm.warm_start = o.warm_start;
    prm.panel_keep = o.panel_l2_keep;
    prm.primal_weight = o.primal_weight;
    prm.queue = nullptr;
    return prm;
}

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
    return sms > 0 ? sms : 148;
}

template <class M, class S>
int run(const ff_problem* probs, int count, const ff_options& o, void* ws, size_t ws_bytes, ff_result* res,
        void* const* w_out, void* const* yA_out, void* const* yD_out, cudaStream_t stream) {
    std::vector<Sizes> sz(count);
    size_t need = table_bytes<M, S>(count);
    for (int t = 0; t < count; ++t) {
        sz[t] = sizes_of(probs[t], o.precision);
        if (!supported(sz[t], probs[t].omega_diag, o.precision)) return FF_ERR_UNSUPPORTED;
        need += inst_bytes(sz[t], probs[t].omega_diag, o.precision);
    }
    if (!ws || ((uintptr_t)ws % kAlign) != 0 || ws_bytes < need) return FF_ERR_WORKSPACE;
    // cluster size per instance, then groups of equal cluster size (largest
    // first); inside a group the largest work comes first in the queue
    std::vector<int> G;
    if (o.cluster_size > 0) G.assign(count, o.cluster_size);
    else choose_clusters(sz, o.cta_work, sm_count(), G);
    auto work = [&](int t) { return (long long)sz[t].n * sz[t].P * (sz[t].k + sz[t].m + 16); };
    std::vector<int> order(count);
    for (int t = 0; t < count; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (G[a] != G[b]) return G[a] > G[b];
        if (sz[a].multi != sz[b].multi) return sz[a].multi > sz[b].multi;
        return work(a) > work(b);
    });
    unsigned char* base = (unsigned char*)ws;
    // table region: count Inst records, count ff_problem records (slot order), queue counters
    Inst<M, S>* table_dev = (Inst<M, S>*)base;
    ff_problem* probs_dev = (ff_problem*)(base + a256((size_t)count * sizeof(Inst<M, S>)));
    int* queue_dev = (int*)(base + a256((size_t)count * sizeof(Inst<M, S>)) + a256((size_t)count * sizeof(ff_problem)));
    unsigned char* cur = base + table_bytes<M, S>(count);
    std::vector<unsigned char> staging(table_bytes<M, S>(count) - kQueueBytes);
    Inst<M, S>* table = (Inst<M, S>*)staging.data();
    ff_problem* pslot = (ff_problem*)(staging.data() + a256((size_t)count * sizeof(Inst<M, S>)));
    long long maxel = 1;
    for (int slot = 0; slot < count; ++slot) {
        int t = order[slot];
        table[slot] = carve<M, S>(probs[t], sz[t], cur, w_out[t], yA_out ? yA_out[t] : nullptr,
                                  yD_out ? yD_out[t] : nullptr, res + t);
        pslot[slot] = probs[t];
        maxel = std::max(maxel, std::max((long long)sz[t].tl.ntile * sz[t].tl.Rp * sz[t].tl.CS,
                                         (long long)sz[t].np * (sz[t].P + sz[t].R)));
    }
    // groups: [first slot, end slot) of equal G and kind (single- or
    // multi-period), at most kMaxGroups
    int gfirst[kMaxGroups + 1], gG[kMaxGroups], ng = 0;
    bool gsingle[kMaxGroups];
    for (int slot = 0; slot < count; ++slot) {
        const int g = G[order[slot]];
        const bool single = !sz[order[slot]].multi;
        if (ng == 0 || gG[ng - 1] != g || gsingle[ng - 1] != single) {
            if (ng == kMaxGroups) return FF_ERR_INVALID_ARG;
            gfirst[ng] = slot;
            gG[ng] = g;
            gsingle[ng] = single;
            ++ng;
        }
    }
    gfirst[ng] = count;
    // shared memory and teams of every group (a group whose cluster cannot be
    // resident falls back to half the cluster size)
    size_t gsmem[kMaxGroups];
    int gteams[kMaxGroups];
    cudaError_t e = cudaSuccess;
    for (int gi = 0; gi < ng; ++gi) {
        size_t smem = 0;
        for (int slot = gfirst[gi]; slot < gfirst[gi + 1]; ++slot) {
            const int t = order[slot];
            smem = std::max(smem, smem_of(sz[t], o.precision));
        }
        int maxc = 0;
        for (;;) {
            e = max_teams<M, S>(gG[gi], smem, gsingle[gi], &maxc);
            if (e != cudaSuccess) return cuda_fail(e, "occupancy query of the solver kernel");
            if (maxc >= 1 || gG[gi] == 1 || o.cluster_size > 0) break;
            gG[gi] /= 2;
        }
        if (maxc < 1) return FF_ERR_UNSUPPORTED;
        int nteams = std::min(gfirst[gi + 1] - gfirst[gi], maxc);
        if (o.max_teams > 0) nteams = std::min(nteams, o.max_teams);
        gsmem[gi] = smem;
        gteams[gi] = nteams;
    }
    if (o.reuse_workspace != 1 && o.reuse_workspace != 2) {
        e = cudaMemcpyAsync(base, staging.data(), staging.size(), cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e, "copy of the instance table");
    }
    if (o.reuse_workspace != 1) {
        const int bx = (int)std::min<long long>(64, (maxel + 255) / 256);
        repack_batch_kernel<M, S><<<dim3((unsigned)bx, (unsigned)count), 256, 0, stream>>>(
            probs_dev, table_dev, (o.precision == FF_PREC_F64 && o.round_panels_bf16) ? 1 : 0);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "repack launch");
    }
    e = cudaMemsetAsync(queue_dev, 0, kQueueBytes, stream);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    Params prm = make_params(o);
    if (ng == 1) {
        prm.queue = queue_dev;
        e = launch_solver<M, S>(table_dev, count, prm, gG[0], gteams[0], gsmem[0], gsingle[0], stream);
        if (e != cudaSuccess) return cuda_fail(e, "solver launch");
        return FF_OK;
    }
    // several groups: one launch each on its own side stream, forked from and
    // joined back into the caller's stream
    std::lock_guard<std::mutex> lock(g_streams_mu);
    DeviceStreams* ds = nullptr;
    int rc = device_streams(&ds);
    if (rc != FF_OK) return rc;
    e = cudaEventRecord(ds->fork, stream);
    if (e != cudaSuccess) return cuda_fail(e, "fork event");
    for (int gi = 0; gi < ng; ++gi) {
        // group 0 has the largest clusters and takes the highest-priority stream
        cudaStream_t sst = ds->side[gi];
        e = cudaStreamWaitEvent(sst, ds->fork, 0);
        if (e != cudaSuccess) return cuda_fail(e, "fork wait");
        prm.queue = queue_dev + gi;
        e = launch_solver<M, S>(table_dev + gfirst[gi], gfirst[gi + 1] - gfirst[gi], prm, gG[gi], gteams[gi],
                                gsmem[gi], gsingle[gi], sst);
        if (e != cudaSuccess) return cuda_fail(e, "solver launch");
        e = cudaEventRecord(ds->join[gi], sst);
        if (e != cudaSuccess) return cuda_fail(e, "join event");
        e = cudaStreamWaitEvent(stream, ds->join[gi], 0);
        if (e != cudaSuccess) return cuda_fail(e, "join wait");
    }
    return FF_OK;
}

int dispatch(const ff_problem* probs, int count, const ff_options* o_in, void* ws, size_t ws_bytes,
             ff_result* res, void* const* w_out, void* const* yA_out, void* const* yD_out, void* stream) {
    if (count < 1 || !probs || !res || !w_out) return FF_ERR_INVALID_ARG;
    if (count > 65535) return FF_ERR_UNSUPPORTED;   // one grid row per instance in the repack launch
    ff_options o;
    if (o_in) o = *o_in; else fill_defaults(&o);
    if (!valid_options(o)) return FF_ERR_INVALID_ARG;
    for (int t = 0; t < count; ++t) {
        if (!valid_problem(&probs[t]) || !w_out[t]) return FF_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    switch (o.precision) {
        case FF_PREC_F64:
            return run<double, double>(probs, count, o, ws, ws_bytes, res, w_out, yA_out, yD_out, st);
        case FF_PREC_F32:
            return run<float, float>(probs, count, o, ws, ws_bytes, res, w_out, yA_out, yD_out, st);
        default:
            return run<float, __nv_bfloat16>(probs, count, o, ws, ws_bytes, res, w_out, yA_out, yD_out, st);
    }
}

// ---------------------------------------------------------------------------
// ff_solve_single_static: the single-period solve on a workspace that lives in
// this library's own device memory (g_static_ws below), for callers that must
// not allocate.  Nothing here allocates: the instance record and the problem
// record reach the array as kernel parameters (store_records_kernel), and the
// workspace address comes from cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
constexpr size_t c_a256(size_t x) { return (x + 255) / 256 * 256; }

std::mutex g_static_mu;
void* g_static_ptr[kMaxStaticDevices] = {};

// Device address of g_static_ws on the current device, looked up once per
// device with that device current.  Returns nullptr (and records the CUDA
// error) when the lookup fails.
void* static_workspace() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { cuda_fail(e, "cudaGetDevice"); return nullptr; }
    if (dev < 0 || dev >= kMaxStaticDevices) {
        snprintf(g_last_error, sizeof(g_last_error), "device ordinal %d beyond the %d supported", dev,
                 kMaxStaticDevices);
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_ws);
        if (e != cudaSuccess) { cuda_fail(e, "cudaGetSymbolAddress of the static workspace"); return nullptr; }
        g_static_ptr[dev] = ptr;
    }
    return g_static_ptr[dev];
}

// Writes the instance record and the problem record into device memory; they
// travel as kernel parameters, so no host buffer has to outlive the call.
template <class M, class S>
__global__ void store_records_kernel(Inst<M, S>* inst_dst, Inst<M, S> inst, ff_problem* prob_dst, ff_problem prob) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *inst_dst = inst;
        *prob_dst = prob;
    }
}

template <class M, class S>
int run_single_static(const ff_problem& p, const ff_options& o, ff_result* res, void* w_out, void* yA_out,
                      void* yD_out, cudaStream_t stream) {
    const Sizes sz = sizes_of(p, o.precision);
    if (!supported(sz, p.omega_diag, o.precision)) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "problem shape not supported by the kernels (n %d, k %d, m %d)", p.n, p.k, p.m);
        return FF_ERR_UNSUPPORTED;
    }
    constexpr size_t kInstBytes = c_a256(sizeof(Inst<M, S>));
    constexpr size_t kStage = kInstBytes + c_a256(sizeof(ff_problem));
    const size_t need = kStage + kQueueBytes + inst_bytes(sz, p.omega_diag, o.precision);
    if (need > (size_t)FF_STATIC_WORKSPACE_BYTES) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "problem needs %zu bytes of workspace; the static workspace holds %zu", need,
                 (size_t)FF_STATIC_WORKSPACE_BYTES);
        return FF_ERR_WORKSPACE;
    }
    // cluster size as ff_solve_single chooses it (cta_work, then spread over
    // the SMs), halved while such a cluster cannot be resident; decided
    // before anything is enqueued
    std::vector<int> Gv;
    if (o.cluster_size > 0) Gv.assign(1, o.cluster_size);
    else choose_clusters(std::vector<Sizes>(1, sz), o.cta_work, sm_count(), Gv);
    int G = Gv[0];
    const size_t smem = smem_of(sz, o.precision);
    int maxc = 0;
    for (;;) {
        cudaError_t e = max_teams<M, S>(G, smem, true, &maxc);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy query of the solver kernel");
        if (maxc >= 1 || G == 1 || o.cluster_size > 0) break;
        G /= 2;
    }
    if (maxc < 1) {
        snprintf(g_last_error, sizeof(g_last_error),
                 "a cluster of %d CTAs with %zu bytes of shared memory each cannot be resident", G, smem);
        return FF_ERR_UNSUPPORTED;
    }
    unsigned char* base = (unsigned char*)static_workspace();
    if (!base) return FF_ERR_CUDA;
    unsigned char* cur = base + kStage + kQueueBytes;
    const Inst<M, S> inst = carve<M, S>(p, sz, cur, w_out, yA_out, yD_out, res);
    Inst<M, S>* table_dev = (Inst<M, S>*)base;
    ff_problem* prob_dev = (ff_problem*)(base + kInstBytes);
    // every region the solver reads is written here, by the repack or by the
    // solver's own initialisation, so nothing has to be cleared between calls
    store_records_kernel<M, S><<<1, 32, 0, stream>>>(table_dev, inst, prob_dev, p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "record store launch");
    long long maxel = std::max((long long)sz.tl.ntile * sz.tl.Rp * sz.tl.CS, (long long)sz.np * (sz.P + sz.R));
    const int bx = (int)std::min<long long>(64, (maxel + 255) / 256);
    repack_batch_kernel<M, S><<<dim3((unsigned)std::max(bx, 1), 1u), 256, 0, stream>>>(
        prob_dev, table_dev, (o.precision == FF_PREC_F64 && o.round_panels_bf16) ? 1 : 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "repack launch");
    int* queue_dev = (int*)(base + kStage);
    e = cudaMemsetAsync(queue_dev, 0, kQueueBytes, stream);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    Params prm = make_params(o);
    prm.queue = queue_dev;
    e = launch_solver<M, S>(table_dev, 1, prm, G, 1, smem, true, stream);
    if (e != cudaSuccess) return cuda_fail(e, "solver launch");
    return FF_OK;
}

int solve_single_static(const ff_problem* p, const ff_options* o_in, ff_result* res, void* w_out, void* yA_out,
                        void* yD_out, void* stream) {
    if (!p || p->T != 0 || !res || !w_out) return FF_ERR_INVALID_ARG;
    ff_options o;
    if (o_in) o = *o_in; else fill_defaults(&o);
    if (!valid_options(o) || !valid_problem(p)) return FF_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    switch (o.precision) {
        case FF_PREC_F64: return run_single_static<double, double>(*p, o, res, w_out, yA_out, yD_out, st);
        case FF_PREC_F32: return run_single_static<float, float>(*p, o, res, w_out, yA_out, yD_out, st);
        default: return run_single_static<float, __nv_bfloat16>(*p, o, res, w_out, yA_out, yD_out, st);
    }
}

}  // namespace
}  // namespace ff

extern "C" {

void ff_default_options(ff_options* o) {
    if (o) ff::fill_defaults(o);
}

size_t ff_joint_workspace_size(const ff_problem* probs, int count) {
    if (!probs || count < 1) return 0;
    for (int t = 0; t < count; ++t)
        if (!ff::valid_problem(&probs[t])) return 0;
    return ff::joint_workspace_bytes(probs, count);
}

int ff_solve_joint_batch(const ff_problem* probs, int count, const ff_options* o_in, void* ws, size_t ws_bytes,
                         ff_result* result_dev, void* const* w_out, void* const* yA_out, void* const* yD_out,
                         void* stream) {
    if (!probs || count < 1 || count > 65535 || !result_dev || !w_out) return FF_ERR_INVALID_ARG;
    ff_options o;
    if (o_in) {
        o = *o_in;
    } else {
        ff::fill_defaults(&o);
        o.precision = FF_PREC_F64;   // the variant's only precision
    }
    if (!ff::valid_options(o)) return FF_ERR_INVALID_ARG;
    if (o.precision != FF_PREC_F64) return FF_ERR_UNSUPPORTED;
    for (int t = 0; t < count; ++t)
        if (!ff::valid_problem(&probs[t])) return FF_ERR_INVALID_ARG;
    cudaError_t ce = cudaSuccess;
    const int rc = ff::joint_solve(probs, count, ff::make_params(o), ws, ws_bytes, result_dev, w_out, yA_out, yD_out,
                                   (cudaStream_t)stream, &ce);
    if (rc == FF_ERR_CUDA) ff::cuda_fail(ce, "joint prox solve (instance table copy or kernel launch)");
    return rc;
}

size_t ff_workspace_size(const ff_problem* probs, int count, const ff_options* o_in) {
    if (!probs || count < 1) return 0;
    ff_options o;
    if (o_in) o = *o_in; else ff::fill_defaults(&o);
    if (!ff::valid_options(o)) return 0;
    size_t need = ff::table_bytes_of(o.precision, count);
    for (int t = 0; t < count; ++t) {
        if (!ff::valid_problem(&probs[t])) return 0;
        need += ff::inst_bytes(ff::sizes_of(probs[t], o.precision), probs[t].omega_diag, o.precision);
    }
    return need;
}

int ff_solve_single(const ff_problem* p, const ff_options* o, void* ws, size_t ws_bytes, ff_result* result_dev,
                    void* w_out, void* yA_out, void* yD_out, void* stream) {
    if (!p || p->T != 0) return FF_ERR_INVALID_ARG;
    void* wo[1] = {w_out};
    void* ya[1] = {yA_out};
    void* yd[1] = {yD_out};
    return ff::dispatch(p, 1, o, ws, ws_bytes, result_dev, wo, ya, yd, stream);
}

int ff_solve_multi(const ff_problem* p, const ff_options* o, void* ws, size_t ws_bytes, ff_result* result_dev,
                   void* w_out, void* yA_out, void* yD_out, void* stream) {
    if (!p || p->T < 2) return FF_ERR_INVALID_ARG;
    void* wo[1] = {w_out};
    void* ya[1] = {yA_out};
    void* yd[1] = {yD_out};
    return ff::dispatch(p, 1, o, ws, ws_bytes, result_dev, wo, ya, yd, stream);
}

int ff_solve_batch(const ff_problem* probs, int count, const ff_options* o, void* ws, size_t ws_bytes,
                   ff_result* result_dev, void* const* w_out, void* const* yA_out, void* const* yD_out,
                   void* stream) {
    return ff::dispatch(probs, count, o, ws, ws_bytes, result_dev, w_out, yA_out, yD_out, stream);
}

int ff_batch_plan(const ff_problem* probs, int count, const ff_options* o_in, int32_t* cluster_out,
                  int32_t* launches_out) {
    if (count < 1 || !probs) return FF_ERR_INVALID_ARG;
    ff_options o;
    if (o_in) o = *o_in; else ff::fill_defaults(&o);
    if (!ff::valid_options(o)) return FF_ERR_INVALID_ARG;
    std::vector<ff::Sizes> sz(count);
    for (int t = 0; t < count; ++t) {
        if (!ff::valid_problem(&probs[t])) return FF_ERR_INVALID_ARG;
        sz[t] = ff::sizes_of(probs[t], o.precision);
    }
    std::vector<int> G;
    if (o.cluster_size > 0) G.assign(count, o.cluster_size);
    else ff::choose_clusters(sz, o.cta_work, ff::sm_count(), G);
    int distinct[32] = {0}, nd = 0;
    for (int t = 0; t < count; ++t) {
        if (cluster_out) cluster_out[t] = G[t];
        const int key = 2 * G[t] + (sz[t].multi ? 1 : 0);
        bool seen = false;
        for (int i = 0; i < nd; ++i) seen = seen || distinct[i] == key;
        if (!seen) distinct[nd++] = key;
    }
    if (launches_out) *launches_out = nd;
    return FF_OK;
}

int ff_solve_single_static(const ff_problem* p, const ff_options* o, ff_result* result_dev, void* w_out,
                           void* yA_out, void* yD_out, void* stream) {
    return ff::solve_single_static(p, o, result_dev, w_out, yA_out, yD_out, stream);
}

const char* ff_status_string(int code) {
    switch (code) {
        case FF_OK: return "ok";
        case FF_ERR_INVALID_ARG: return "invalid argument";
        case FF_ERR_CUDA: return "CUDA runtime error";
        case FF_ERR_WORKSPACE: return "workspace too small or misaligned";
        case FF_ERR_UNSUPPORTED: return "problem shape not supported by the kernels";
        case FF_ERR_DEVICE: return "device-side error flag set";
        default: return "unknown status";
    }
}

int ff_version(void) { return 300; }   // 0.3.0: ff_options and ff_result fields appended, risk model, joint prox

const char* ff_last_error(void) { return ff::g_last_error; }

}  // extern "C"
