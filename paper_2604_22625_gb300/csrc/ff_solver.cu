// Persistent "team" kernel: one thread-block cluster of G CTAs solves one
// portfolio instance at a time (single-period model, Sec. 2.1, or
// multi-period model, Sec. 2.2) and then takes the next instance of the batch
// from a device queue (largest first, so the tail is short).
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
// Steps: tau = 2 s / L_f and sum_i sigma_i ||K_i||^2 = 1/tau - beta L_f with
// beta > 1/2, reflection rho <= (2 beta - 1) / (2 beta).
//
// Precision: panels F, A stored as S and multiplied in M (FP32 or FP64),
// tile sums added in FP64.  The iterate state (x, x0, y, y0) is FP64.  In the
// FP32/BF16 modes (M = float) each iteration's changes are computed as FP32
// increments of FP64 differences (the step u = -tau (grad f + K^T y), the
// projection x_bar - x, the Halpern combination, the trade residuals and the
// dual update) and applied to the FP64 state; the l1 threshold search compares
// in FP32 and sums as double-float pairs.  The FP64 mode keeps every operation
// in FP64.  The KKT evaluation is FP64 in all modes.
//
// Work split inside a team: CTA g owns the assets [i0, i1).  Two passes over
// the panels per iteration:
//   expand (thread per asset, factor-major F^T and A):  F (Omega u), A^T y_A
//   reduce (thread per row, asset-major F and A^T):     A x_bar, A x_new, F^T x_new
// Sums over assets across the CTAs of the cluster go through distributed
// shared memory (each CTA adds one slice over all ranks in fixed order and
// writes it back to every rank), so every CTA holds bit-identical totals and
// takes identical control-flow decisions.  All waits are hardware cluster
// barriers; there is no spin loop.
#include <cooperative_groups.h>
#include <math.h>

#include <type_traits>

#include "ff_internal.cuh"

namespace cg = cooperative_groups;

namespace ff {

// ---------------------------------------------------------------------------
// shared-memory layout (identical on host and device)
// ---------------------------------------------------------------------------
struct Layout {
    size_t vpart, vout;        // double, vlen each (one chunk of periods; vpart also holds the
                               // expand pass's cross-split partial sums)
    size_t spart, sout;        // double, slen each
    size_t wred;               // double, kWarps * 32
    size_t stage;              // M, 4 vectors x PCT periods x CH assets (reduce pass)
    size_t yA, yAb, ax;        // double, P*m each
    size_t u, ub;              // double, P*k each
    size_t om;                 // M, P*k
    size_t yAm;                // M, P*m
    size_t Om;                 // double, k*k or k
    size_t cand, thprev, theta, thq;
    size_t lb, ubd;            // double, m each
    size_t bars;               // kStages mbarriers
    size_t vbuf;               // double, vcap (single period, v in shared memory)
    size_t ring;               // kStages panel tiles
    size_t panel_bytes;        // panel tile bytes within a stage (128-aligned)
    size_t tile_bytes;         // stage stride
    size_t total;
    int vlen, slen;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// rep_glob = 1: the per-period replicated arrays yA, yAb, ax, u, ub live in a
// per-CTA slice of the workspace instead of shared memory (many periods in
// FP64, where they would not leave room for a panel tile)
__host__ __device__ inline Layout make_layout(int P, int k, int m, int omega_diag, size_t ms, int CH, int Rp,
                                              size_t ps, int vcap, int rep_glob = 0) {
    Layout L;
    const int pct0 = P < kPC ? P : kPC;
    const int pct = pct0 <= 1 ? 1 : (pct0 <= 2 ? 2 : (pct0 <= 4 ? 4 : 8));   // template chunk width
    L.vlen = pct0 * (2 * m + 2 * k);
    const int slots = (kWarps * P * kCand + 1) / 2;   // 4-byte threshold slots in 8-byte units
    if (L.vlen < slots) L.vlen = slots;
    // the expand pass's cross-split partials (kThreads x 2 x pct, up to double)
    // occupy vpart and vout together
    if (L.vlen < kThreads * pct) L.vlen = kThreads * pct;
    int s1 = P * kCand * 2, s2 = P + 48;
    L.slen = s1 > s2 ? s1 : s2;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes + 16, 16); return r; };
    L.bars = take((size_t)kStages * 8);   // first: the barriers keep their place across instances
    L.vpart = take((size_t)L.vlen * 8);
    L.vout = take((size_t)L.vlen * 8);
    L.spart = take((size_t)L.slen * 8);
    L.sout = take((size_t)L.slen * 8);
    L.wred = take((size_t)kWarps * 32 * 8);
    L.stage = take((size_t)4 * pct * CH * (ms > 8 ? ms : 8));   // staged as M, or double at checks
    // whole chunks for the expand pass weights (a single period needs no padding)
    const int Pr = P <= 1 ? 1 : (P + kPC - 1) / kPC * kPC;
    const int rs = rep_glob ? 0 : 1;
    L.yA = take((size_t)rs * P * m * 8);
    L.yAb = take((size_t)rs * Pr * m * 8);
    L.ax = take((size_t)rs * P * m * 8);
    L.u = take((size_t)rs * P * k * 8);
    L.ub = take((size_t)rs * Pr * k * 8);
    L.om = take((size_t)Pr * k * ms);
    L.yAm = take((size_t)Pr * m * ms);
    L.Om = take((size_t)(omega_diag ? k : k * k) * 8);
    L.cand = take((size_t)P * kCand * 8);
    L.thprev = take((size_t)P * 8);
    L.theta = take((size_t)P * 8);
    L.thq = take((size_t)P * 8);
    L.lb = take((size_t)m * 8);
    L.ubd = take((size_t)m * 8);
    L.vbuf = take((size_t)vcap * 8);
    o = align_up(o, 128);
    // one stage: the panel tile, then (single period) the per-asset vectors that
    // the fused passes stage with it: 5 FP64 (x, x0, yD, yD0, w0) + 2 M (c1, c2)
    L.panel_bytes = align_up((size_t)Rp * tile_stride(CH, (int)ps) * ps, 128);
    L.tile_bytes = L.panel_bytes + (P == 1 ? align_up((size_t)CH * (5 * 8 + 2 * ms), 128) : 0);
    L.ring = o;
    o += (size_t)kStages * L.tile_bytes;
    L.total = o;
    return L;
}

size_t solver_smem_bytes(int P, int k, int m, int omega_diag, size_t matvec_size, int CH, int Rp,
                         size_t panel_size, int vcap, int rep_glob) {
    return make_layout(P, k, m, omega_diag, matvec_size, CH, Rp, panel_size, vcap, rep_glob).total;
}

int choose_tile(int P, int n, int k, int m, int omega_diag, size_t matvec_size, size_t panel_size, int* vcap,
                int* rep_glob) {
    const int Rp = (k + 7) / 8 * 8 + (m + 7) / 8 * 8;
    // the single-period variant is built for kSingleCtasPerSm resident CTAs
    const size_t limit = P == 1 ? (size_t)kSmemLimit / kSingleCtasPerSm - 1024 : (size_t)kSmemLimit;
    const size_t max_tile = P == 1 ? (size_t)kMaxTileBytes / kSingleCtasPerSm : (size_t)kMaxTileBytes;
    // passes: v in shared memory (single period), everything in shared memory,
    // per-period replicated arrays in the workspace (multi-period)
    for (int pass = (P == 1 ? 0 : 1); pass < 3; ++pass) {
        if (pass == 2 && P == 1) break;
        const int rg = pass == 2 ? 1 : 0;
        for (int CH = 256; CH >= 8; CH /= 2) {
            if ((size_t)Rp * tile_stride(CH, (int)panel_size) * panel_size > max_tile) continue;
            // the replicated arrays move to the workspace only when the tile
            // would otherwise be narrower than 32 assets
            if (pass == 1 && P > 1 && CH < 32) break;
            const int vc = pass == 0 ? (n + CH - 1) / CH * CH : 0;
            if (make_layout(P, k, m, omega_diag, matvec_size, CH, Rp, panel_size, vc, rg).total <= limit) {
                *vcap = vc;
                *rep_glob = rg;
                return CH;
            }
        }
    }
    *vcap = 0;
    *rep_glob = 0;
    return 0;
}

// ---------------------------------------------------------------------------
// bulk-copy ring: one thread issues cp.async.bulk copies of whole panel tiles
// into kStages shared-memory stages, each completing on its own mbarrier.
// Every thread keeps an identical copy of the ring state (all follow the same
// sequence of waits), so stage indices and phase parities need no sharing.
// ---------------------------------------------------------------------------
struct Pipe {
    unsigned char* ring;
    unsigned long long* bars;
    size_t stride;            // bytes per stage (the instance's tile bytes, 128-aligned)
    int head;                 // next stage to consume
    int tail;                 // next stage to fill
    int inflight;             // copies issued and not yet consumed
    unsigned phase;           // bit s: parity of the phase stage s completes next
    int* err;                 // shared flag: a bounded wait expired
    int frozen;               // after an expired wait: no copy is issued and no phase flipped
                              // until pipe_drain has let the copies in flight land
    int waits;                // waits of the current instance (the test hook expires the first)
    int expire_first;         // test hook: treat the instance's first wait as expired
    int keep;                 // 1: panel tiles carry an L2 evict_last policy
    unsigned long long policy;   // the L2 cache policy of the panel tiles (keep = 1)
};

// A panel-tile copy: with keep, the L2 policy asks to keep the panel's lines
// (an instance re-reads its panel twice per iteration); per-asset vectors are
// copied with the default policy.
__device__ __forceinline__ void bulk_copy(unsigned dst, const void* src, unsigned bytes, unsigned bar, int keep,
                                          unsigned long long policy) {
    if (keep)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
            ::"r"(dst), "l"(src), "r"(bytes), "r"(bar), "l"(policy)
            : "memory");
    else
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                     : "memory");
}

constexpr int kWaitSpins = 1 << 22;    // try_wait polls of one wait before it counts as expired

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// thread 0 of the CTA initialises the barriers (once per kernel)
__device__ __forceinline__ void pipe_init(Pipe& pp) {
    if (threadIdx.x == 0) {
        for (int s2 = 0; s2 < kStages; ++s2)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&pp.bars[s2])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

// Issue the copy of `bytes` from global `src` into the tail stage.  Called by
// every thread (uniform), performed by thread 0.  A frozen ring issues nothing.
__device__ __forceinline__ void pipe_issue(Pipe& pp, const void* src, unsigned bytes) {
    if (pp.frozen) return;
    if (threadIdx.x == 0) {
        const unsigned bar = smem_u32(&pp.bars[pp.tail]);
        const unsigned dst = smem_u32(pp.ring + (size_t)pp.tail * pp.stride);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        bulk_copy(dst, src, bytes, bar, pp.keep, pp.policy);
    }
    pp.tail = pp.tail + 1 == kStages ? 0 : pp.tail + 1;
    ++pp.inflight;
}

// Issue nc copies into the tail stage that complete on its one barrier:
// copy q moves bytes[q] from src[q] to the stage offset off[q].
__device__ __forceinline__ void pipe_issue_n(Pipe& pp, int nc, const void* const* src, const unsigned* off,
                                             const unsigned* bytes) {
    if (pp.frozen) return;
    if (threadIdx.x == 0) {
        unsigned total = 0;
        for (int q = 0; q < nc; ++q) total += bytes[q];
        const unsigned bar = smem_u32(&pp.bars[pp.tail]);
        unsigned char* stage = pp.ring + (size_t)pp.tail * pp.stride;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(total) : "memory");
        for (int q = 0; q < nc; ++q)   // copy 0 is the panel tile
            bulk_copy(smem_u32(stage + off[q]), src[q], bytes[q], bar, q == 0 ? pp.keep : 0, pp.policy);
    }
    pp.tail = pp.tail + 1 == kStages ? 0 : pp.tail + 1;
    ++pp.inflight;
}

// Poll the barrier of stage `st` for the phase of parity `parity`, at most
// `spins` times; true once that phase has completed.
__device__ __forceinline__ bool bar_poll(const Pipe& pp, int st, unsigned parity, int spins) {
    const unsigned bar = smem_u32(&pp.bars[st]);
    unsigned done = 0;
    for (int spin = 0; spin < spins; ++spin) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) break;
    }
    return done != 0;
}

// Wait (bounded) until the head stage has landed; returns its shared address.
// On expiry the shared error flag is set and the stage is used as it is; the
// next pipe_pop then freezes the ring (the instance ends with FF_STALLED at its
// next check, which every CTA of the team takes together).  A frozen ring
// returns at once: its data are not used for a result.
__device__ __forceinline__ const unsigned char* pipe_wait(Pipe& pp) {
    const unsigned char* stage = pp.ring + (size_t)pp.head * pp.stride;
    if (pp.frozen) return stage;
    const bool expire = pp.expire_first && pp.waits == 0;
    ++pp.waits;
    if (expire || !bar_poll(pp, pp.head, (pp.phase >> pp.head) & 1u, kWaitSpins)) *pp.err = 1;
    return stage;
}

// The head stage has been read by every thread (caller synchronised, so every
// thread sees the same error flag): move on.  After an expired wait the ring
// freezes instead: the stage's phase is not flipped (its copy may still be
// landing), so the bookkeeping keeps matching the barriers for pipe_drain.
__device__ __forceinline__ void pipe_pop(Pipe& pp) {
    if (pp.frozen) return;
    if (*pp.err) { pp.frozen = 1; return; }
    pp.phase ^= 1u << pp.head;
    pp.head = pp.head + 1 == kStages ? 0 : pp.head + 1;
    --pp.inflight;
}

// Before the team leaves an instance: let every copy still in flight land
// (bounded waits on the phases the bookkeeping expects) and unfreeze the
// ring.  Copies of valid global memory complete in microseconds, so the bound
// is only reached on a hardware fault; the return value (false then) is the
// same on every thread of the CTA.
__device__ bool pipe_drain(Pipe& pp) {
    bool ok = true;
    while (pp.inflight > 0) {
        ok = bar_poll(pp, pp.head, (pp.phase >> pp.head) & 1u, kWaitSpins) && ok;
        pp.phase ^= 1u << pp.head;
        pp.head = pp.head + 1 == kStages ? 0 : pp.head + 1;
        --pp.inflight;
    }
    pp.frozen = 0;
    return __syncthreads_and(ok ? 1 : 0) != 0;
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float cvt(float a) { return a; }
__device__ __forceinline__ double cvt(double a) { return a; }
__device__ __forceinline__ float cvt(__nv_bfloat16 a) { return __bfloat162float(a); }

template <class A, class S>
__device__ __forceinline__ A ldp(const S* p) { return (A)cvt(__ldg(p)); }

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Scalar prox of gamma * (c1 |z| + c2 |z|^d) at t (Sec. 2.1 cost, one asset), FP64.
__device__ __forceinline__ double prox_cost(double t, double gamma, double c1, double c2, double d) {
    double a = fabs(t) - gamma * c1;
    if (!(a > 0.0)) return 0.0;
    double r;
    double gc = gamma * c2;
    if (gc <= 0.0) {
        r = a;
    } else if (d == 1.5) {
        // r + 1.5 gc sqrt(r) = a  ->  rho = sqrt(r) solves rho^2 + beta rho - a = 0
        double beta = 1.5 * gc;
        double rho = 2.0 * a / (beta + sqrt(beta * beta + 4.0 * a));
        r = rho * rho;
    } else if (d == 2.0) {
        r = a / (1.0 + 2.0 * gc);
    } else {
        // safeguarded Newton on h(r) = r + gc d r^(d-1) - a over [0, a]
        double lo = 0, hi = a;
        r = a;
        for (int it = 0; it < 80; ++it) {
            double rp = pow(r, d - 1.0);
            double h = r + gc * d * rp - a;
            if (h > 0) hi = r; else lo = r;
            double dh = 1.0 + gc * d * (d - 1.0) * (r > 0 ? rp / r : 0.0);
            double rn = r - h / dh;
            if (!(rn > lo && rn < hi)) rn = 0.5 * (lo + hi);
            if (fabs(rn - r) <= 1e-16 * a) { r = rn; break; }
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

// Dual update of one trade row (Moreau identity for h_D(v) = phi(v + b)):
//   t = p / sigma + b,  z = prox_{phi / sigma}(t),  y = sigma (t - z).
// On the live branch (|t| > c1 / sigma) y = phi'(z) = sign(t) (c1 + d c2 |z|^(d-1)),
// evaluated in M without the cancellation of p - sigma (z - b); in the dead zone
// y = sigma t = p + sigma b exactly.  Returns true on the live branch.
template <class M>
__device__ __forceinline__ bool trade_multiplier(double t, double inv_sigma, double c1d, double c2d, double d,
                                                 M& y_live) {
    const M c1 = (M)c1d, c2 = (M)c2d;
    const M g = (M)inv_sigma;
    const M tm = (M)t;
    const M a = fabs(tm) - g * c1;
    if (!(a > (M)0)) return false;
    M deriv;
    const M gc = g * c2;
    if (gc <= (M)0) {
        deriv = c1;
    } else if (d == 1.5) {
        // z = rho^2 with rho^2 + beta rho - a = 0, beta = 1.5 g c2: phi'(z) = c1 + 1.5 c2 rho
        const M beta = (M)1.5 * gc;
        const M rho = (M)2 * a / (beta + sqrt(beta * beta + (M)4 * a));
        deriv = c1 + (M)1.5 * c2 * rho;
    } else if (d == 2.0) {
        deriv = c1 + (M)2 * c2 * (a / ((M)1 + (M)2 * gc));
    } else {
        // general exponent: FP64 safeguarded Newton for |z|, derivative in M
        const M r = (M)fabs(prox_cost(t, inv_sigma, c1d, c2d, d));
        deriv = c1 + (M)d * c2 * (M)pow((double)r, d - 1.0);
    }
    y_live = tm < 0 ? -deriv : deriv;
    return true;
}

// The multiplier form in FP32 throughout (t, 1/sigma, c1, c2 already FP32):
// returns true on the live branch with y = phi'(z) in y_live.
__device__ __forceinline__ bool trade_multiplier_f(float t, float g, float c1, float c2, double d, float& y_live) {
    const float a = fabsf(t) - g * c1;
    if (!(a > 0.f)) return false;
    float deriv;
    const float gc = g * c2;
    if (gc <= 0.f) {
        deriv = c1;
    } else if (d == 1.5) {
        const float beta = 1.5f * gc;
        const float rho = 2.f * a / (beta + sqrtf(beta * beta + 4.f * a));
        deriv = c1 + 1.5f * c2 * rho;
    } else if (d == 2.0) {
        deriv = c1 + 2.f * c2 * (a / (1.f + 2.f * gc));
    } else {
        const double r = fabs(prox_cost((double)t, (double)g, (double)c1, (double)c2, d));
        deriv = c1 + (float)(d * (double)c2 * pow(r, d - 1.0));
    }
    y_live = t < 0.f ? -deriv : deriv;
    return true;
}

// ---------------------------------------------------------------------------
// per-CTA context
// ---------------------------------------------------------------------------
template <class M, class S>
struct Ctx {
    Inst<M, S> I;
    int n, k, m, P, R, np;
    int i0, i1;
    int t0, t1;                // panel tiles of this CTA
    unsigned panel_off;        // offset of the per-asset vectors within a stage
    int G, g;
    Pipe pipe;
    int tid, lane, warp;
    double *vpart, *vout, *spart, *sout, *wred;
    M* stage;
    double *yA, *yAb, *ax, *u, *ub, *Om, *lb, *ubd;
    M *om, *yAm;
    double *cand, *thprev, *theta, *thq;
};

// Sum (or max) of part[0..K) over the team; result in out[0..K) of every CTA.
// The G remote loads of an entry are issued together and added in rank order,
// so every CTA receives bit-identical totals.
// Entries [0, ksum) are summed, entries [ksum, K) take the maximum.
__device__ void team_reduce_mixed(cg::cluster_group& cl, double* part, double* out, int K, int ksum, int G, int g) {
    cl.sync();
    const int per = (K + G - 1) / G;
    const int lo = g * per;
    const int hi = min(K, lo + per);
    for (int idx = lo + (int)threadIdx.x; idx < hi; idx += blockDim.x) {
        const bool mx = idx >= ksum;
        double v[kMaxCluster];
#pragma unroll
        for (int q = 0; q < kMaxCluster; ++q)
            if (q < G) v[q] = cl.map_shared_rank(part, q)[idx];
        double s = v[0];
#pragma unroll
        for (int q = 1; q < kMaxCluster; ++q)
            if (q < G) s = mx ? fmax(s, v[q]) : s + v[q];
        for (int q = 0; q < G; ++q) cl.map_shared_rank(out, q)[idx] = s;
    }
    cl.sync();
}

template <bool MAX>
__device__ void team_reduce(cg::cluster_group& cl, double* part, double* out, int K, int G, int g) {
    cl.sync();
    const int per = (K + G - 1) / G;
    const int lo = g * per;
    const int hi = min(K, lo + per);
    for (int idx = lo + (int)threadIdx.x; idx < hi; idx += blockDim.x) {
        double v[kMaxCluster];
#pragma unroll
        for (int q = 0; q < kMaxCluster; ++q)
            if (q < G) v[q] = cl.map_shared_rank(part, q)[idx];
        double s = v[0];
#pragma unroll
        for (int q = 1; q < kMaxCluster; ++q)
            if (q < G) s = MAX ? fmax(s, v[q]) : s + v[q];
        for (int q = 0; q < G; ++q) cl.map_shared_rank(out, q)[idx] = s;
    }
    cl.sync();
}

// Block-wide sum (or max) of NV doubles held by every thread; thread i < NV
// writes dst[i].  Ends with __syncthreads.  (Used outside the inner loop.)
template <int NV, bool MAX = false>
__device__ void block_reduce(double (&v)[NV], double* dst, double* wred, int lane, int warp) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double w = __shfl_xor_sync(0xffffffffu, v[i], o);
            v[i] = MAX ? fmax(v[i], w) : v[i] + w;
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) wred[warp * 32 + i] = v[i];
    }
    __syncthreads();
    if ((int)threadIdx.x < NV) {
        double s = MAX ? -INFINITY : 0.0;
        for (int w = 0; w < kWarps; ++w)
            s = MAX ? fmax(s, wred[w * 32 + threadIdx.x]) : s + wred[w * 32 + threadIdx.x];
        dst[threadIdx.x] = s;
    }
    __syncthreads();
}

// error-free float transformations (Knuth TwoSum) for double-float warp sums
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_add(float& hi, float& lo, float bhi, float blo) {
    float s, e;
    two_sum(hi, bhi, s, e);
    e += lo + blo;
    hi = s + e;
    lo = e - (hi - s);
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Double-float state of the FP32/BF16 modes: a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi) / 2 (about 48 bits), kept in a
// float2 in the slot of a double.  The iteration changes it only by FP32
// increments, so every update is one error-free add; differences of two
// nearby states are exact in their hi parts (Sterbenz) and carry the lo parts,
// so FP32 work keeps the accuracy of the former FP64 state without FP64
// instructions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 df_split(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}
__device__ __forceinline__ double df_value(float2 a) { return (double)a.x + (double)a.y; }
// a + b (b an FP32 increment), renormalised
__device__ __forceinline__ float2 df_inc(float2 a, float b) {
    const float s = a.x + b;
    const float bb = s - a.x;
    const float e = (a.x - (s - bb)) + (b - bb) + a.y;
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}
// a - b rounded to FP32 (a, b close: the hi difference is exact)
__device__ __forceinline__ float df_sub(float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); }

// ---------------------------------------------------------------------------
// reduce pass over one chunk of periods [p0, p0 + pc), pc <= PCT:
//   vpart[q*Lr + j]          = sum_i A_ji a0_{p0+q, i}          (j < m)
//   vpart[q*Lr + m + j]      = sum_i A_ji a1_{p0+q, i}
//   vpart[q*Lr + 2m + j]     = sum_i F_ij (f0_{p0+q, i} - c_i)   (j < k)
//   vpart[q*Lr + 2m + k + j] = sum_i F_ij (f1_{p0+q, i} - c_i)
// with Lr = 2m + 2k, over the CTA's assets.  The panel tiles stream through the
// bulk-copy ring; the vectors of a tile are staged in shared memory as M while
// its copy is in flight.  Thread mapping: groups of na consecutive threads own
// 4 consecutive panel rows, the na lanes of a group take every na-th asset of
// the tile (the padded row stride keeps the groups on distinct banks).  Products and per-tile sums in M (at most CH / na terms), lanes
// combined by warp shuffles, tile sums added into vpart in FP64 by the group's
// first lane (one owner per entry: no races, fixed order).  Null vectors give
// zeros.
// ---------------------------------------------------------------------------
// Products of one panel tile with the staged vectors.  sv0A/sv1A feed the A
// rows, sv0F/sv1F the F rows ([PCT][CH] each).  The products accumulate in
// acc (AT, per thread) across consecutive tiles; reduce_flush combines the
// lanes of each row group by shuffles and adds the sums into vpart in FP64
// (one owner per entry, fixed order) and clears acc.
template <int PCT, class AT> struct ReduceAcc {
    AT a[4][2][PCT];
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < PCT; ++q) { a[r][0][q] = 0; a[r][1][q] = 0; }
    }
};

struct ReduceMap {
    int na, grp, lane_a, r0;
    bool active, isA;
};

template <class M, class S>
__device__ __forceinline__ ReduceMap reduce_map(const Ctx<M, S>& c) {
    constexpr int RPT = 4;
    ReduceMap mp;
    const int ngr = c.I.Rp / RPT;
    int na = 1;
    while (na < 32 && ngr * na * 2 <= kThreads) na *= 2;
    mp.na = na;
    mp.grp = c.tid / na;
    mp.lane_a = c.tid % na;
    mp.active = mp.grp < ngr;
    mp.r0 = mp.grp * RPT;
    mp.isA = mp.r0 >= c.I.kp;
    return mp;
}

template <int PCT, class AT, class M, class S>
__device__ __forceinline__ void reduce_tile(Ctx<M, S>& c, const ReduceMap& mp, ReduceAcc<PCT, AT>& acc,
                                            const S* tile, const AT* sv0A, const AT* sv1A, const AT* sv0F,
                                            const AT* sv1F, int cnt, bool has1) {
    constexpr int RPT = 4;
    const int CH = c.I.CH, CS = c.I.CS;
    if (mp.active) {
        const AT* sv0 = mp.isA ? sv0A : sv0F;
        const AT* sv1 = mp.isA ? sv1A : sv1F;
        const S* rows = tile + (size_t)mp.r0 * CS;
        for (int ii = mp.lane_a; ii < cnt; ii += mp.na) {
            AT w[RPT];
#pragma unroll
            for (int r = 0; r < RPT; ++r) w[r] = (AT)cvt(rows[(size_t)r * CS + ii]);
#pragma unroll
            for (int q = 0; q < PCT; ++q) {
                const AT x0 = sv0[q * CH + ii];
                const AT x1 = has1 ? sv1[q * CH + ii] : (AT)0;
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    acc.a[r][0][q] += w[r] * x0;
                    acc.a[r][1][q] += w[r] * x1;
                }
            }
        }
    }
}

template <int PCT, class AT, class M, class S>
__device__ __forceinline__ void reduce_flush(Ctx<M, S>& c, const ReduceMap& mp, ReduceAcc<PCT, AT>& acc, int pc) {
    constexpr int RPT = 4;
    const int kp = c.I.kp, m = c.m, k = c.k;
    const int Lr = 2 * m + 2 * k;
    for (int off = mp.na / 2; off > 0; off >>= 1) {
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int q = 0; q < PCT; ++q) {
                acc.a[r][0][q] += __shfl_xor_sync(0xffffffffu, acc.a[r][0][q], off);
                acc.a[r][1][q] += __shfl_xor_sync(0xffffffffu, acc.a[r][1][q], off);
            }
    }
    if (mp.active && mp.lane_a == 0) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int row = mp.r0 + r;
            int o0 = -1, o1 = -1;
            if (!mp.isA && row < k) { o0 = 2 * m + row; o1 = 2 * m + k + row; }
            if (mp.isA && row - kp < m) { o0 = row - kp; o1 = m + row - kp; }
            if (o0 >= 0) {
#pragma unroll
                for (int q = 0; q < PCT; ++q) {
                    if (q < pc) {
                        c.vpart[q * Lr + o0] += (double)acc.a[r][0][q];
                        c.vpart[q * Lr + o1] += (double)acc.a[r][1][q];
                    }
                }
            }
        }
    }
    acc.clear();
}

constexpr int kFlushTiles = 4;   // tiles summed in the matvec precision before an FP64 flush

template <int PCT, class AT, class M, class S>
__device__ void reduce_chunk_t(Ctx<M, S>& c, int p0, int pc, const double* a0, const double* a1,
                               const double* f0, const double* f1, bool subcen) {
    const int CH = c.I.CH, Rp = c.I.Rp;
    const int m = c.m, k = c.k, np = c.np, n = c.n;
    const int Lr = 2 * m + 2 * k;
    const bool has1 = (a1 != nullptr) || (f1 != nullptr);
    (void)CH;
    // the F-row vectors are the A-row vectors (no centre, same arrays): stage two
    const bool single_fa = !c.I.multi && a0 != nullptr && a1 != nullptr && f0 == a1 && (f1 == nullptr || f1 == a0);
    const size_t tile_elems = (size_t)Rp * c.I.CS;
    const unsigned bytes = (unsigned)(tile_elems * sizeof(S));
    AT* st = (AT*)c.stage;  // [4][PCT][CH]
    for (int e = c.tid; e < pc * Lr; e += kThreads) c.vpart[e] = 0;
    const ReduceMap mp = reduce_map(c);
    ReduceAcc<PCT, AT> acc;
    acc.clear();
    const int nt = c.t1 - c.t0;
    for (int j = 0; j < nt && j < kStages; ++j) pipe_issue(c.pipe, c.I.PE + (size_t)(c.t0 + j) * tile_elems, bytes);
    for (int j = 0; j < nt; ++j) {
        const int t = c.t0 + j;
        const int ib = t * CH;
        const int cnt = min(CH, n - ib);
        // single period (centre 0): the F rows take the same two vectors as the
        // A rows, in swapped roles (f0 = a1, f1 = a0), so only two are staged
        const int nvec = single_fa ? 2 : 4;
        for (int e = c.tid; e < nvec * PCT * CH; e += kThreads) {
            const int vec = e / (PCT * CH);
            const int q = (e / CH) % PCT;
            const int ii = e % CH;
            double val = 0;
            const double* src = vec == 0 ? a0 : vec == 1 ? a1 : vec == 2 ? f0 : f1;
            if (src && q < pc && ii < cnt) {
                const int i = ib + ii;
                val = src[(size_t)(p0 + q) * np + i] - ((subcen && vec >= 2) ? c.I.cen[i] : 0.0);
            }
            st[e] = (AT)val;
        }
        const S* tile = (const S*)pipe_wait(c.pipe);
        __syncthreads();
        reduce_tile<PCT, AT>(c, mp, acc, tile, st, st + PCT * CH, st + (single_fa ? 1 : 2) * PCT * CH,
                             st + (single_fa ? 0 : 3) * PCT * CH, cnt, has1);
        if ((j + 1) % kFlushTiles == 0 || j + 1 == nt) reduce_flush<PCT, AT>(c, mp, acc, pc);
        __syncthreads();
        pipe_pop(c.pipe);
        if (j + kStages < nt) pipe_issue(c.pipe, c.I.PE + (size_t)(t + kStages) * tile_elems, bytes);
    }
    __syncthreads();
}

// Multi-period reduce pass of the FP32-increment iteration: the staged vectors
// come from the pair buffer (x_bar, x+) in FP32: A rows take (x_bar, x+), F
// rows (x+ - c, x_bar - c).
template <int PCT, class M, class S>
__device__ void reduce_pairs_t(Ctx<M, S>& c, int p0, int pc, const float2* vp) {
    const int CH = c.I.CH, Rp = c.I.Rp;
    const int m = c.m, k = c.k, np = c.np, n = c.n;
    const int Lr = 2 * m + 2 * k;
    const size_t tile_elems = (size_t)Rp * c.I.CS;
    const unsigned bytes = (unsigned)(tile_elems * sizeof(S));
    float* st = (float*)c.stage;  // [4][PCT][CH]
    for (int e = c.tid; e < pc * Lr; e += kThreads) c.vpart[e] = 0;
    const ReduceMap mp = reduce_map(c);
    ReduceAcc<PCT, float> acc;
    acc.clear();
    const int nt = c.t1 - c.t0;
    for (int j = 0; j < nt && j < kStages; ++j) pipe_issue(c.pipe, c.I.PE + (size_t)(c.t0 + j) * tile_elems, bytes);
    for (int j = 0; j < nt; ++j) {
        const int t = c.t0 + j;
        const int ib = t * CH;
        const int cnt = min(CH, n - ib);
        for (int e = c.tid; e < PCT * CH; e += kThreads) {
            const int q = e / CH, ii = e % CH;
            float xb = 0.f, xn = 0.f, cf = 0.f;
            if (q < pc && ii < cnt) {
                const int i = ib + ii;
                const float2 pr = vp[(size_t)(p0 + q) * np + i];
                xb = pr.x;
                xn = pr.y;
                cf = c.I.cenf[i];
            }
            st[e] = xb;
            st[PCT * CH + e] = xn;
            st[2 * PCT * CH + e] = xn - cf;
            st[3 * PCT * CH + e] = xb - cf;
        }
        const S* tile = (const S*)pipe_wait(c.pipe);
        __syncthreads();
        reduce_tile<PCT, float>(c, mp, acc, tile, st, st + PCT * CH, st + 2 * PCT * CH, st + 3 * PCT * CH, cnt,
                                true);
        if ((j + 1) % kFlushTiles == 0 || j + 1 == nt) reduce_flush<PCT, float>(c, mp, acc, pc);
        __syncthreads();
        pipe_pop(c.pipe);
        if (j + kStages < nt) pipe_issue(c.pipe, c.I.PE + (size_t)(t + kStages) * tile_elems, bytes);
    }
    __syncthreads();
}

template <class M, class S>
__device__ void reduce_chunk_pairs(Ctx<M, S>& c, int p0, int pc, const float2* vp) {
    if (pc <= 1) reduce_pairs_t<1>(c, p0, pc, vp);
    else if (pc <= 2) reduce_pairs_t<2>(c, p0, pc, vp);
    else if (pc <= 4) reduce_pairs_t<4>(c, p0, pc, vp);
    else reduce_pairs_t<8>(c, p0, pc, vp);
}

// ---------------------------------------------------------------------------
// Single-period fused pass (elementwise prox + Halpern + reduce): each panel tile
// arrives together with its assets' x, x0, y_D, y_D0, w0 (FP64) and c1, c2
// (M) in one stage.  For the tile's assets the threads form
//   x_bar = Proj(v) (threshold theta),  x+ = hlA x_bar + hlB x + hlC x0,
//   y_bar = sigma-prox of the trade cost at y + sigma (2 x_bar - x),  y+ likewise,
// write x+ and y+ (and, at checks, x_bar and y_bar) to the workspace, stage
// x_bar and x+ as M, and the panel products of the tile follow:
//   A x_bar, A x+ (A rows);  F^T x+, F^T x_bar (F rows; no centre).
// ---------------------------------------------------------------------------
template <class M, class S>
__device__ void reduce_fused_single(Ctx<M, S>& c, double hlA, double hlB, double hlC, double sD, double inv_sD,
                                    double dexp, bool check, double (&rloc)[2]) {
    const int CH = c.I.CH, Rp = c.I.Rp;
    const int m = c.m, k = c.k, n = c.n, np = c.np;
    const int Lr = 2 * m + 2 * k;
    const size_t tile_elems = (size_t)Rp * c.I.CS;
    const unsigned pbytes = (unsigned)(tile_elems * sizeof(S));
    const unsigned po = c.panel_off;
    const unsigned off[8] = {0u, po, po + 8u * CH, po + 16u * CH, po + 24u * CH, po + 32u * CH, po + 40u * CH,
                             po + 40u * CH + (unsigned)sizeof(M) * CH};
    M* st = c.stage;  // [2][CH]: x_bar, x+
    const double theta = c.theta[0];
    // FP32 copies of the pass's scalars, converted once (not per element)
    const float fA = (float)hlA, fC = (float)hlC, fsD = (float)sD, finv = (float)inv_sD, th = (float)theta;
    for (int e = c.tid; e < Lr; e += kThreads) c.vpart[e] = 0;
    const ReduceMap mp = reduce_map(c);
    ReduceAcc<1, M> acc;
    acc.clear();
    auto issue = [&](int t) {
        const int ib = t * CH;
        const unsigned nv = (unsigned)min(CH, np - ib);
        const void* w0src = std::is_same<M, float>::value ? (const void*)(c.I.w0f + ib) : (const void*)(c.I.w0 + ib);
        const void* src[8] = {c.I.PE + (size_t)t * tile_elems, c.I.x + ib, c.I.x0 + ib, c.I.yD + ib, c.I.yD0 + ib,
                              w0src, c.I.c1 + ib, c.I.c2 + ib};
        const unsigned bytes[8] = {pbytes, 8u * nv, 8u * nv, 8u * nv, 8u * nv, 8u * nv, (unsigned)sizeof(M) * nv,
                                   (unsigned)sizeof(M) * nv};
        pipe_issue_n(c.pipe, 8, src, off, bytes);
    };
    const int nt = c.t1 - c.t0;
    for (int j = 0; j < nt && j < kStages; ++j) issue(c.t0 + j);
    for (int j = 0; j < nt; ++j) {
        const int t = c.t0 + j;
        const int ib = t * CH;
        const int cnt = min(CH, n - ib);
        const unsigned char* stg = pipe_wait(c.pipe);
        const S* tile = (const S*)stg;
        const double* sx = (const double*)(stg + off[1]);
        const double* sx0 = (const double*)(stg + off[2]);
        const double* syd = (const double*)(stg + off[3]);
        const double* syd0 = (const double*)(stg + off[4]);
        const double* sw0 = (const double*)(stg + off[5]);
        const M* sc1 = (const M*)(stg + off[6]);
        const M* sc2 = (const M*)(stg + off[7]);
        for (int ii = c.tid; ii < cnt; ii += kThreads) {
            const int i = ib + ii;
            if constexpr (std::is_same<M, float>::value) {
                // FP32 increments on the double-float state (see the multi-period pass)
                const float2 vu = ((const float2*)c.I.v)[i];
                const float2 xc = ((const float2*)sx)[ii];
                const float av = fabsf(vu.x) - th;
                float d1, xbf = 0.f;
                if (av > 0.f) {
                    d1 = vu.y - (vu.x < 0.f ? -th : th);
                    xbf = vu.x < 0.f ? -av : av;
                } else {
                    d1 = -(xc.x + xc.y);
                }
                const float2 xn = df_inc(xc, fA * d1 + fC * df_sub(((const float2*)sx0)[ii], xc));
                const float zz = df_sub(xc, ((const float2*)sw0)[ii]) + 2.f * d1;   // (x - w0) + 2 (x_bar - x)
                const float2 yd = ((const float2*)syd)[ii];
                const float ydf = yd.x;
                const float tf = ydf * finv + zz;
                float yl, dy;
                if (trade_multiplier_f(tf, finv, sc1[ii], sc2[ii], dexp, yl)) dy = (yl - yd.x) - yd.y;
                else dy = fsD * zz;
                ((float2*)c.I.xn)[i] = xn;
                ((float2*)c.I.yDn)[i] = df_inc(yd, fA * dy + fC * df_sub(((const float2*)syd0)[ii], yd));
                if (check) {
                    c.I.xb[i] = av > 0.f ? df_value(xc) + (double)d1 : 0.0;   // exact zeros off the support
                    c.I.yDb[i] = df_value(yd) + (double)dy;
                    rloc[0] += (double)d1 * (double)d1;
                    rloc[1] += (double)dy * (double)dy;
                }
                st[ii] = xbf;
                st[CH + ii] = xn.x;
            } else {
                const double vv = c.I.v[i];
                const double av = fabs(vv) - theta;
                const double xb = av > 0 ? (vv < 0 ? -av : av) : 0.0;
                const double xc = sx[ii];
                const double xn = hlA * xb + hlB * xc + hlC * sx0[ii];
                const double dxe = 2.0 * xb - xc;          // (Delta (2 x_bar - x))_1
                const double b = -sw0[ii];
                const double yd = syd[ii];
                const double pD = yd + sD * dxe;
                const double tt = pD * inv_sD + b;
                M ylive;
                const double ydb = trade_multiplier<M>(tt, inv_sD, (double)sc1[ii], (double)sc2[ii], dexp, ylive)
                                       ? (double)ylive
                                       : pD + sD * b;
                const double ydn = hlA * ydb + hlB * yd + hlC * syd0[ii];
                c.I.xn[i] = xn;
                c.I.yDn[i] = ydn;
                if (check) {
                    c.I.xb[i] = xb;
                    c.I.yDb[i] = ydb;
                    rloc[0] += (xc - xb) * (xc - xb);
                    rloc[1] += (yd - ydb) * (yd - ydb);
                }
                st[ii] = (M)xb;
                st[CH + ii] = (M)xn;
            }
        }
        __syncthreads();
        // A rows: (x_bar, x+); F rows: (x+, x_bar)
        reduce_tile<1, M>(c, mp, acc, tile, st, st + CH, st + CH, st, cnt, true);
        if ((j + 1) % kFlushTiles == 0 || j + 1 == nt) reduce_flush<1, M>(c, mp, acc, 1);
        __syncthreads();
        pipe_pop(c.pipe);
        if (j + kStages < nt) issue(t + kStages);
    }
    // the x+ / y+ written here are read by bulk copies (async proxy) next iteration
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
}

// PCMAX = 1: the kernel variant for single-period instances (only the
// one-period code is instantiated, which keeps its register count low)
// AT: arithmetic of the products and tile sums (M, or double for the FP64
// pass of the KKT check)
template <int PCMAX, class AT = void, class M, class S>
__device__ void reduce_chunk(Ctx<M, S>& c, int p0, int pc, const double* a0, const double* a1, const double* f0,
                             const double* f1, bool subcen) {
    using T = typename std::conditional<std::is_same<AT, void>::value, M, AT>::type;
    if constexpr (PCMAX == 1) {
        reduce_chunk_t<1, T>(c, p0, pc, a0, a1, f0, f1, subcen);
    } else {
        if (pc <= 1) reduce_chunk_t<1, T>(c, p0, pc, a0, a1, f0, f1, subcen);
        else if (pc <= 2) reduce_chunk_t<2, T>(c, p0, pc, a0, a1, f0, f1, subcen);
        else if (pc <= 4) reduce_chunk_t<4, T>(c, p0, pc, a0, a1, f0, f1, subcen);
        else reduce_chunk_t<8, T>(c, p0, pc, a0, a1, f0, f1, subcen);
    }
}

// FP64 reduce of the KKT check in chunks of at most 4 periods: its
// accumulator (4 rows x 2 vectors x PCT doubles per thread) would otherwise
// take 128 registers at PCT = 8 and force spills in the multi-period variant
template <int PCMAX, class M, class S>
__device__ void reduce_chunk_f64(Ctx<M, S>& c, int p0, int pc, const double* f1) {
    if (pc <= 1) reduce_chunk_t<1, double>(c, p0, pc, nullptr, nullptr, nullptr, f1, true);
    else if (pc <= 2) reduce_chunk_t<2, double>(c, p0, pc, nullptr, nullptr, nullptr, f1, true);
    else reduce_chunk_t<4, double>(c, p0, pc, nullptr, nullptr, nullptr, f1, true);
}

// ---------------------------------------------------------------------------
// expand pass: for every local asset i and period p < Pv,
//   epi(i, p, (F wF_p)_i, (A^T wA_p)_i)     with wF (Pv x k), wA (Pv x m)
// arithmetic in A (M or double).  The PE tiles ([Rp][CH], assets contiguous)
// stream through the bulk-copy ring.  Thread mapping inside a tile: asset
// ii = tid % CH, row split rs = tid / CH (RS = kThreads / CH splits, each a
// contiguous share of the F rows and of the A rows); the splits' partial sums
// meet in shared memory (vpart..vout) and the (asset, period) epilogues are
// spread over all threads.
// ---------------------------------------------------------------------------
template <int PCT, class A, class M, class S, class W, class Epi>
__device__ void expand_tile(Ctx<M, S>& c, const S* tile, int ib, int cnt, int p0, int pc, const W* wF,
                            const W* wA, Epi& epi) {
    const int CH = c.I.CH, CS = c.I.CS, kp = c.I.kp, k = c.k, m = c.m;
    const int RS = kThreads / CH;
    const int ii = c.tid % CH, rs = c.tid / CH;
    A aF[PCT], aA[PCT];
#pragma unroll
    for (int q = 0; q < PCT; ++q) { aF[q] = 0; aA[q] = 0; }
    const W* wf = wF + (size_t)p0 * k;
    const W* wa = wA + (size_t)p0 * m;
    const int jf0 = k * rs / RS, jf1 = k * (rs + 1) / RS;
    const int ja0 = m * rs / RS, ja1 = m * (rs + 1) / RS;
    int j = jf0;
    for (; j + 4 <= jf1; j += 4) {
        A f[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) f[u] = (A)cvt(tile[(size_t)(j + u) * CS + ii]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < PCT; ++q) aF[q] += f[u] * (A)wf[q * k + j + u];
    }
    for (; j < jf1; ++j) {
        const A f = (A)cvt(tile[(size_t)j * CS + ii]);
#pragma unroll
        for (int q = 0; q < PCT; ++q) aF[q] += f * (A)wf[q * k + j];
    }
    j = ja0;
    for (; j + 4 <= ja1; j += 4) {
        A a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = (A)cvt(tile[(size_t)(kp + j + u) * CS + ii]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < PCT; ++q) aA[q] += a[u] * (A)wa[q * m + j + u];
    }
    for (; j < ja1; ++j) {
        const A a = (A)cvt(tile[(size_t)(kp + j) * CS + ii]);
#pragma unroll
        for (int q = 0; q < PCT; ++q) aA[q] += a * (A)wa[q * m + j];
    }
    if (RS == 1) {
        if (ii < cnt) {
#pragma unroll
            for (int q = 0; q < PCT; ++q)
                if (q < pc) epi(ib + ii, p0 + q, aF[q], aA[q]);
        }
        return;
    }
    A* red = (A*)c.vpart;   // [RS][CH][2][PCT]
#pragma unroll
    for (int q = 0; q < PCT; ++q) {
        red[(((size_t)rs * CH + ii) * 2 + 0) * PCT + q] = aF[q];
        red[(((size_t)rs * CH + ii) * 2 + 1) * PCT + q] = aA[q];
    }
    __syncthreads();
    for (int e = c.tid; e < CH * pc; e += kThreads) {
        const int i2 = e % CH, q = e / CH;
        if (i2 < cnt) {
            A sF = 0, sA = 0;
            for (int r = 0; r < RS; ++r) {
                sF += red[(((size_t)r * CH + i2) * 2 + 0) * PCT + q];
                sA += red[(((size_t)r * CH + i2) * 2 + 1) * PCT + q];
            }
            epi(ib + i2, p0 + q, sF, sA);
        }
    }
    __syncthreads();
}

// The weight vectors must have PCT rows readable past Pv: callers size the
// replicated arrays for whole chunks (rows beyond Pv hold finite values).
template <class A, int PCMAX, class M, class S, class W, class Epi>
__device__ void expand_pass(Ctx<M, S>& c, int Pv, const W* wF, const W* wA, Epi epi) {
    const int CH = c.I.CH;
    const size_t tile_elems = (size_t)c.I.Rp * c.I.CS;
    const unsigned bytes = (unsigned)(tile_elems * sizeof(S));
    const int nt = c.t1 - c.t0;
    for (int j = 0; j < nt && j < kStages; ++j) pipe_issue(c.pipe, c.I.PE + (size_t)(c.t0 + j) * tile_elems, bytes);
    for (int j = 0; j < nt; ++j) {
        const int t = c.t0 + j;
        const int ib = t * CH;
        const int cnt = min(CH, c.n - ib);
        const S* tile = (const S*)pipe_wait(c.pipe);
        if constexpr (PCMAX == 1) {
            expand_tile<1, A>(c, tile, ib, cnt, 0, 1, wF, wA, epi);
        } else {
            for (int p0 = 0; p0 < Pv; p0 += kPC) {
                const int pc = min(kPC, Pv - p0);
                if (pc <= 1) expand_tile<1, A>(c, tile, ib, cnt, p0, pc, wF, wA, epi);
                else if (pc <= 2) expand_tile<2, A>(c, tile, ib, cnt, p0, pc, wF, wA, epi);
                else if (pc <= 4) expand_tile<4, A>(c, tile, ib, cnt, p0, pc, wF, wA, epi);
                else expand_tile<8, A>(c, tile, ib, cnt, p0, pc, wF, wA, epi);
            }
        }
        __syncthreads();
        pipe_pop(c.pipe);
        if (j + kStages < nt) pipe_issue(c.pipe, c.I.PE + (size_t)(t + kStages) * tile_elems, bytes);
    }
}

// Single-period main expand pass: the PE tile arrives with its assets' x, y_D
// (FP64) and alpha, D (M) in one stage; v = x - tau (grad f(x) + K^T y).
template <class M, class S>
__device__ void expand_main_single(Ctx<M, S>& c, double tau, double kap, const M* wF, const M* wA) {
    const int CH = c.I.CH, Rp = c.I.Rp;
    const int n = c.n, np = c.np;
    const size_t tile_elems = (size_t)Rp * c.I.CS;
    const unsigned pbytes = (unsigned)(tile_elems * sizeof(S));
    const unsigned po = c.panel_off;
    const unsigned off[5] = {0u, po, po + 8u * CH, po + 16u * CH, po + 16u * CH + (unsigned)sizeof(M) * CH};
    const M kapm = (M)kap;
    const float ftau = (float)tau;
    double* v = c.I.v;
    auto issue = [&](int t) {
        const int ib = t * CH;
        const unsigned nv = (unsigned)min(CH, np - ib);
        const void* src[5] = {c.I.PE + (size_t)t * tile_elems, c.I.x + ib, c.I.yD + ib, c.I.alpha + ib,
                              c.I.Dp + ib};
        const unsigned bytes[5] = {pbytes, 8u * nv, 8u * nv, (unsigned)sizeof(M) * nv, (unsigned)sizeof(M) * nv};
        pipe_issue_n(c.pipe, 5, src, off, bytes);
    };
    const int nt = c.t1 - c.t0;
    for (int j = 0; j < nt && j < kStages; ++j) issue(c.t0 + j);
    for (int j = 0; j < nt; ++j) {
        const int t = c.t0 + j;
        const int ib = t * CH;
        const int cnt = min(CH, n - ib);
        const unsigned char* stg = pipe_wait(c.pipe);
        const S* tile = (const S*)stg;
        const double* sx = (const double*)(stg + off[1]);
        const double* syd = (const double*)(stg + off[2]);
        const M* sal = (const M*)(stg + off[3]);
        const M* sdp = (const M*)(stg + off[4]);
        auto epi = [&](int i, int p, auto aF, auto aA) {
            const int ii = i - ib;
            const double xv = sx[ii];
            if constexpr (std::is_same<M, float>::value) {
                // FP32 step u and v = x + u as a pair (the FP32-increment iteration);
                // x and y_D are double-float pairs: their hi parts suffice here
                const float xf = ((const float2*)sx)[ii].x;
                const float gf = -sal[ii] + 2.f * kapm * ((float)aF + sdp[ii] * xf);
                const float kt = (float)aA + ((const float2*)syd)[ii].x;
                const float u = -ftau * (gf + kt);
                ((float2*)v)[i] = make_float2(xf + u, u);
            } else {
                const M gf = -sal[ii] + (M)2 * kapm * ((M)aF + sdp[ii] * (M)xv);
                const M kt = (M)aA + (M)syd[ii];
                v[i] = xv - tau * (double)(gf + kt);
            }
        };
        expand_tile<1, M>(c, tile, ib, cnt, 0, 1, wF, wA, epi);
        __syncthreads();
        pipe_pop(c.pipe);
        if (j + kStages < nt) issue(t + kStages);
    }
}

// ---------------------------------------------------------------------------
// l1-ball projection thresholds for every period of vector vv (P x np):
// theta_p >= 0 with S(theta) = sum_i max(|v_pi| - theta, 0) = 1, or 0 when
// ||v_p||_1 <= 1 (projection onto the budget set of Eq. 3 / Eq. 6).
// S is convex, decreasing and piecewise linear with breakpoints at the |v_i|.
// Newton's method from the warm start t_0:
//   t_{k+1} = (sum_{|v| > t_k} |v| - 1) / #{|v| > t_k}
// lands at or below the root from any start (tangents of a convex function
// lie below it).  When the count #{|v| > t} is the same at t_k and t_{k+1},
// no breakpoint lies between them, S is linear there and t_{k+1} is the
// root exactly.  FP64 sums; warp sums as error-free double-float pairs; the
// per-warp partials are added in warp order (deterministic).
// Returns the number of rounds (passes over v).
// ---------------------------------------------------------------------------
template <class V, class M, class S>
__device__ int l1_thresholds(cg::cluster_group& cl, Ctx<M, S>& c, const V* vv, double* th_out,
                             double* th_warm) {
    const int P = c.P, np = c.np;
    float* slotS = (float*)c.vpart;     // [kWarps][P][2]  (hi, lo)
    int* slotN = (int*)c.vout;          // [kWarps][P]
    float* slotB = (float*)(slotN + kWarps * P);   // [kWarps][P][2] bracket (max inactive, min active)
    __shared__ int done_s[64];
    __shared__ double t_s[64];
    __shared__ int nprev_s[64];
    for (int p = c.tid; p < P; p += kThreads) {
        done_s[p] = 0;
        t_s[p] = th_warm[p] > 0 ? th_warm[p] : 0.0;
        nprev_s[p] = -1;
    }
    __syncthreads();
    const bool wpp = P >= kWarps / 2;   // one warp per period, else all warps on every period
    const int pstart = wpp ? c.warp : 0;
    const int pstep = wpp ? kWarps : 1;
    const int istart = wpp ? c.i0 + c.lane : c.i0 + c.tid;
    const int istep = wpp ? 32 : kThreads;
    const int nw = wpp ? 1 : kWarps;
    int rounds_done = 0;
    for (int round = 0; round < kMaxRounds; ++round) {
        for (int p = pstart; p < P; p += pstep) {
            if (done_s[p]) continue;
            const V* vp = vv + (size_t)p * np;
            const double t = t_s[p];
            int nd = 0;
            float hi, lo, bl, bh;   // sum pair; bracket: largest |v| <= t, smallest |v| > t
            if constexpr (std::is_same<V, double>::value) {
                double sd = 0, l = -1.0, h = INFINITY;
#pragma unroll 4
                for (int i = istart; i < c.i1; i += istep) {
                    const double a = fabs(vp[i]);
                    if (a > t) { sd += a; nd += 1; h = fmin(h, a); }
                    else l = fmax(l, a);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    l = fmax(l, __shfl_xor_sync(0xffffffffu, l, o));
                    h = fmin(h, __shfl_xor_sync(0xffffffffu, h, o));
                }
                hi = (float)sd;
                lo = (float)(sd - (double)hi);
                bl = __double2float_ru(l);   // rounded outward: the bracket test stays conservative
                bh = __double2float_rd(h);
            } else {
                // FP32 entries (v.x), compared with the rounded threshold and
                // summed as an error-free double-float pair
                const float tf = (float)t;
                hi = 0.f;
                lo = 0.f;
                bl = -1.f;
                bh = INFINITY;
#pragma unroll 4
                for (int i = istart; i < c.i1; i += istep) {
                    const float a = fabsf(vp[i].x);
                    if (a > tf) {
                        float sum, err;
                        two_sum(hi, a, sum, err);
                        hi = sum;
                        lo += err;
                        nd += 1;
                        bh = fminf(bh, a);
                    } else {
                        bl = fmaxf(bl, a);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    bl = fmaxf(bl, __shfl_xor_sync(0xffffffffu, bl, o));
                    bh = fminf(bh, __shfl_xor_sync(0xffffffffu, bh, o));
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float sh = __shfl_xor_sync(0xffffffffu, hi, o);
                const float sl = __shfl_xor_sync(0xffffffffu, lo, o);
                df_add(hi, lo, sh, sl);
            }
            const int nsum = __reduce_add_sync(0xffffffffu, nd);
            if (c.lane == 0) {
                const int slot = wpp ? p : (c.warp * P + p);
                slotS[2 * slot] = hi;
                slotS[2 * slot + 1] = lo;
                slotN[slot] = nsum;
                slotB[2 * slot] = bl;
                slotB[2 * slot + 1] = bh;
            }
        }
        __syncthreads();
        for (int p = c.tid; p < P; p += kThreads) {
            double sv = 0, nn = 0, bl = -1.0, bh = INFINITY;
            if (!done_s[p]) {
                for (int w = 0; w < nw; ++w) {
                    const int slot = wpp ? p : (w * P + p);
                    sv += (double)slotS[2 * slot] + (double)slotS[2 * slot + 1];
                    nn += (double)slotN[slot];
                    bl = fmax(bl, (double)slotB[2 * slot]);
                    bh = fmin(bh, (double)slotB[2 * slot + 1]);
                }
            }
            c.spart[2 * p] = sv;
            c.spart[2 * p + 1] = nn;
            c.spart[2 * P + 2 * p] = bl;
            c.spart[2 * P + 2 * p + 1] = -bh;
        }
        team_reduce_mixed(cl, c.spart, c.sout, 4 * P, 2 * P, c.G, c.g);
        // one thread per period decides (every CTA of the team holds the same sums)
        {
            for (int p = c.tid; p < P; p += kThreads) {
                if (done_s[p]) continue;
                const double Sv = c.sout[2 * p];
                const int Nv = (int)c.sout[2 * p + 1];
                const double t = t_s[p];
                if (t == 0.0 && Sv <= 1.0) {                   // inside the ball
                    th_out[p] = 0.0;
                    done_s[p] = 1;
                    continue;
                }
                if (Nv == nprev_s[p]) {                        // no breakpoint crossed: exact
                    th_out[p] = t;
                    done_s[p] = 1;
                    continue;
                }
                double tn = (Sv - 1.0) / (double)(Nv > 0 ? Nv : 1);
                // the Newton point keeps the active set of t (no |v| between t and
                // tn): S is linear on the bracket and tn is the root, in one pass
                const double blo = c.sout[2 * P + 2 * p], bhi = -c.sout[2 * P + 2 * p + 1];
                const double tcmp = std::is_same<V, double>::value ? tn : (double)(float)tn;
                if (Nv > 0 && tn > 0.0 && blo <= tcmp && tcmp < bhi) {
                    th_out[p] = tn;
                    done_s[p] = 1;
                    continue;
                }
                if (tn <= 0.0) {                               // step from above past 0: test 0
                    tn = 0.0;
                    nprev_s[p] = -1;
                } else {
                    nprev_s[p] = Nv;
                }
                t_s[p] = tn;
                if (round == kMaxRounds - 1) {                 // budget spent: a lower bound
                    th_out[p] = tn;
                    done_s[p] = 1;
                }
            }
        }
        __syncthreads();
        ++rounds_done;
        int rem = 0;
        for (int p = 0; p < P; ++p) rem += done_s[p] ? 0 : 1;
        if (rem == 0) break;
    }
    if (c.tid == 0)
        for (int p = 0; p < P; ++p) th_warm[p] = th_out[p];
    __syncthreads();
    return rounds_done;
}

// om_p = Omega u_p for all periods, written as M (replicated in every CTA)
template <class M, class S>
__device__ void apply_omega_m(Ctx<M, S>& c, const double* uin, M* out, int Pv) {
    const int k = c.k;
    for (int e = c.tid; e < Pv * k; e += kThreads) {
        const int p = e / k, j = e % k;
        double s;
        if (c.I.omega_diag) {
            s = c.Om[j] * uin[p * k + j];
        } else {
            s = 0;
            for (int l = 0; l < k; ++l) s += c.Om[j * k + l] * uin[p * k + l];
        }
        out[e] = (M)s;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <class M, class S, int PCMAX>
__global__ void __launch_bounds__(kThreads, PCMAX == 1 ? kSingleCtasPerSm : 1)
team_kernel(const Inst<M, S>* __restrict__ insts, int count, Params prm) {
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int G = (int)cl.num_blocks();
    const int g = (int)cl.block_rank();
    // FP32 increments on the FP64 state (FP32 and BF16 modes); FP64 mode keeps
    // every elementwise operation in FP64
    constexpr bool kIncr = std::is_same<M, float>::value;
    __shared__ int next_s;
    __shared__ int pipe_err_s;
    __shared__ int ring_broken_s;   // a copy never landed: no further copies on this CTA
    __shared__ int decide_s[2];     // rank 0's decisions at a check: stop status (-1: go on), restart
    Pipe pipe;
    pipe.bars = (unsigned long long*)smem;   // the layout puts the barriers first
    pipe.ring = nullptr;
    pipe.stride = 0;
    pipe.head = 0;
    pipe.tail = 0;
    pipe.inflight = 0;
    pipe.phase = 0;
    pipe.err = &pipe_err_s;
    pipe.frozen = 0;
    pipe.waits = 0;
    pipe.expire_first = prm.expire_first_wait;
    pipe.keep = prm.panel_keep;
    pipe.policy = 0;
    if (prm.panel_keep) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pipe.policy));
    if (threadIdx.x == 0) { pipe_err_s = 0; ring_broken_s = 0; }
    pipe_init(pipe);

    for (;;) {
        // the team's rank-0 thread takes the next instance from the queue and
        // the other ranks read it from rank 0's shared memory
        if (g == 0 && threadIdx.x == 0) next_s = atomicAdd(prm.queue, 1);
        cl.sync();
        const int inst = *cl.map_shared_rank(&next_s, 0);
        cl.sync();
        if (inst >= count) break;
        Ctx<M, S> c;
        c.I = insts[inst];
        c.n = c.I.n; c.k = c.I.k; c.m = c.I.m; c.np = c.I.np;
        c.P = PCMAX == 1 ? 1 : c.I.P;
        c.R = PCMAX == 1 ? 1 : c.I.R;
        c.G = G; c.g = g;
        c.tid = threadIdx.x; c.lane = threadIdx.x & 31; c.warp = threadIdx.x >> 5;
        c.t0 = (int)(((long long)c.I.ntile * g) / G);
        c.t1 = (int)(((long long)c.I.ntile * (g + 1)) / G);
        c.i0 = min(c.n, c.t0 * c.I.CH);
        c.i1 = min(c.n, c.t1 * c.I.CH);
        const int n = c.n, k = c.k, m = c.m, P = c.P, R = c.R, np = c.np;
        const int Lr = 2 * m + 2 * k;
        const Layout Ly = make_layout(P, k, m, c.I.omega_diag, sizeof(M), c.I.CH, c.I.Rp, sizeof(S), c.I.vcap,
                                      c.I.rep_glob);
        // v in shared memory holds this CTA's assets [i0, i1): offset the
        // pointer so that v[i] addresses entry i - i0
        if (PCMAX == 1 && c.I.vcap > 0) c.I.v = (double*)(smem + Ly.vbuf) - c.i0;
        pipe.ring = smem + Ly.ring;
        pipe.stride = Ly.tile_bytes;
        c.pipe = pipe;
        c.pipe.waits = 0;
        c.pipe.frozen = ring_broken_s;   // uniform: written before the last cluster barrier
        c.panel_off = (unsigned)Ly.panel_bytes;
        if (threadIdx.x == 0) pipe_err_s = ring_broken_s;
        c.vpart = (double*)(smem + Ly.vpart);
        c.vout = (double*)(smem + Ly.vout);
        c.spart = (double*)(smem + Ly.spart);
        c.sout = (double*)(smem + Ly.sout);
        c.wred = (double*)(smem + Ly.wred);
        c.stage = (M*)(smem + Ly.stage);
        if (c.I.rep_glob) {
            // this CTA's slice of the workspace (no other CTA touches it)
            const int Pr = P <= 1 ? 1 : (P + kPC - 1) / kPC * kPC;
            double* rb = c.I.rep + (size_t)g * rep_doubles(P, k, m);
            c.yA = rb;
            c.yAb = c.yA + (size_t)P * m;
            c.ax = c.yAb + (size_t)Pr * m;
            c.u = c.ax + (size_t)P * m;
            c.ub = c.u + (size_t)P * k;
        } else {
            c.yA = (double*)(smem + Ly.yA);
            c.yAb = (double*)(smem + Ly.yAb);
            c.ax = (double*)(smem + Ly.ax);
            c.u = (double*)(smem + Ly.u);
            c.ub = (double*)(smem + Ly.ub);
        }
        c.om = (M*)(smem + Ly.om);
        c.yAm = (M*)(smem + Ly.yAm);
        c.Om = (double*)(smem + Ly.Om);
        c.cand = (double*)(smem + Ly.cand);
        c.thprev = (double*)(smem + Ly.thprev);
        c.theta = (double*)(smem + Ly.theta);
        c.thq = (double*)(smem + Ly.thq);
        c.lb = (double*)(smem + Ly.lb);
        c.ubd = (double*)(smem + Ly.ubd);
        const double kap = c.I.kappa;
        const double dexp = c.I.d;
        const unsigned long long t_start = globaltimer();
        double ph[6] = {0, 0, 0, 0, 0, 0};
        unsigned long long tph = t_start;
        auto lap = [&](int slot) {
            const unsigned long long t = globaltimer();
            ph[slot] += (double)(t - tph);
            tph = t;
        };
        long long th_rounds = 0;

        // ---- prologue: replicated constants -------------------------------
        for (int e = c.tid; e < (c.I.omega_diag ? k : k * k); e += kThreads) c.Om[e] = c.I.Om[e];
        for (int e = c.tid; e < m; e += kThreads) { c.lb[e] = c.I.L[e]; c.ubd[e] = c.I.U[e]; }
        __syncthreads();

        // ---- Lipschitz constants by power iteration (M-precision matvecs) ---
        // lambda_max(F Omega F^T + diag(Dmax)) and ||A||^2 = lambda_max(A A^T)
        double lamS = 0, lamA = 0;
        {
            double* v1 = c.I.pv1;
            double* v2 = c.I.pv2;
            for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                const double s = 1.0 + 0.25 * (double)((i * 2654435761u) % 1000u) / 1000.0;
                v1[i] = s;
                v2[i] = s;
            }
            __syncthreads();
            for (int it = 0; it < prm.power_iters; ++it) {
                reduce_chunk<PCMAX>(c, 0, 1, v2, (const double*)nullptr, v1, (const double*)nullptr, false);
                team_reduce<false>(cl, c.vpart, c.vout, Lr, G, g);
                for (int e = c.tid; e < k; e += kThreads) c.u[e] = c.vout[2 * m + e];
                for (int e = c.tid; e < m; e += kThreads) c.yAm[e] = (M)c.vout[e];
                __syncthreads();
                apply_omega_m(c, c.u, c.om, 1);
                double nrm[2] = {0, 0};
                expand_pass<M, PCMAX>(c, 1, c.om, c.yAm, [&](int i, int p, auto aF, auto aA) {
                    const double w1 = aF + c.I.Dmax[i] * v1[i];
                    nrm[0] += w1 * w1;
                    nrm[1] += aA * aA;
                    c.I.xb[i] = w1;
                    c.I.xn[i] = aA;
                });
                block_reduce<2>(nrm, c.spart, c.wred, c.lane, c.warp);
                team_reduce<false>(cl, c.spart, c.sout, 2, G, g);
                // v is a unit vector from the second step on, so ||Sigma v|| -> lambda_max
                const double n1 = sqrt(c.sout[0]), n2 = sqrt(c.sout[1]);
                lamS = n1;
                lamA = n2;
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                    v1[i] = n1 > 0 ? c.I.xb[i] / n1 : 0.0;
                    v2[i] = n2 > 0 ? c.I.xn[i] / n2 : 0.0;
                }
                __syncthreads();
            }
        }
        const double Lf = 2.0 * kap * lamS * 1.05;
        const double nA2 = (m > 0) ? fmax(lamA * 1.05, 1e-300) : 1.0;
        const double nD2 = c.I.multi ? 4.0 : 1.0;
        double tau = prm.step_fraction * 2.0 / Lf;
        // sigma_A ||A||^2 + sigma_D ||Delta||^2 = 1/tau - beta L_f (split evenly): the
        // gradient step is then beta-cocoercive in the step metric, the iteration map
        // is 2 beta / (4 beta - 1)-averaged, and reflection up to (2 beta - 1)/(2 beta)
        // keeps it nonexpansive (Condat 2013, Thm 3.1; averaged-operator calculus)
        const double qsplit = (m > 0) ? 2.0 : 1.0;
        const double sig = (1.0 / tau - prm.beta * Lf) / qsplit;
        double sA = sig / nA2;
        double sD = sig / nD2;
        double inv_sD = 1.0 / sD;
        double inv_sA = 1.0 / sA;
        // Primal weight (adaptive steps, option primal_weight): omega = sqrt(sigma_D / tau),
        // the ratio of the trade-block dual step to the primal step.  At a restart
        // it moves halfway (in logarithm) toward ||dy|| / ||dx||, the distances
        // the dual and the primal iterates travelled in the last cycle (PDLP's
        // rule), and the steps are re-solved from the same budget,
        //   1/tau = beta L_f + s,  sigma_A ||A||^2 + sigma_D ||Delta||^2 = s,
        // with s (beta L_f + s) = omega^2 qsplit ||Delta||^2, so the Condat-Vu
        // step condition keeps holding for every omega.
        const double omega0 = sqrt(sD / tau);
        double omega = omega0;
        auto set_steps = [&](double om) {
            const double bL = prm.beta * Lf;
            const double sv = 0.5 * (-bL + sqrt(bL * bL + 4.0 * om * om * qsplit * nD2));
            tau = 1.0 / (bL + sv);
            sA = sv / (qsplit * nA2);
            sD = sv / (qsplit * nD2);
            inv_sD = 1.0 / sD;
            inv_sA = 1.0 / sA;
        };
        const double rho = prm.rho;

        // ---- initial point: w0 (single) / straight line w0 -> w_T (multi), or
        //      (warm start) the values the output buffers hold ----------------
        auto out_at = [&](const void* buf, size_t idx) -> double {
            return c.I.out_f64 ? ((const double*)buf)[idx] : (double)((const float*)buf)[idx];
        };
        const bool warm = prm.warm_start != 0;
        for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
            const double w0 = c.I.w0[i];
            const double wt = c.I.multi ? c.I.cen[i] : w0;
            for (int p = 0; p < P; ++p) {
                const double x = warm ? out_at(c.I.w_out, (size_t)p * n + i)
                                      : (c.I.multi ? w0 + (wt - w0) * (double)(p + 1) / (double)(P + 1) : w0);
                c.I.x[(size_t)p * np + i] = x;
                c.I.x0[(size_t)p * np + i] = x;
            }
            for (int r = 0; r < R; ++r) {
                const double y = (warm && c.I.yD_out) ? out_at(c.I.yD_out, (size_t)r * n + i) : 0.0;
                c.I.yD[(size_t)r * np + i] = y;
                c.I.yD0[(size_t)r * np + i] = y;
            }
        }
        if constexpr (kIncr && PCMAX != 1) {
            // FP32 views the multi-period expand reads: x in the pair buffer, y_D's FP32 copy
            for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                for (int p = 0; p < P; ++p)
                    ((float2*)c.I.v)[(size_t)p * np + i] = make_float2(0.f, (float)c.I.x[(size_t)p * np + i]);
                for (int r = 0; r < R; ++r) c.I.yDf[(size_t)r * np + i] = (float)c.I.yD[(size_t)r * np + i];
            }
        }
        for (int e = c.tid; e < P * m; e += kThreads) {
            const double y = (warm && c.I.yA_out) ? out_at(c.I.yA_out, (size_t)e) : 0.0;
            c.yA[e] = y;
            c.yAb[e] = y;
            c.yAm[e] = (M)y;
            c.I.yA0[e] = y;
        }
        for (int p = c.tid; p < P; p += kThreads) {
            c.thprev[p] = 0;
            c.thq[p] = 0;
        }
        // the initial iterate is read by bulk copies (async proxy)
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __syncthreads();
        // u = F^T (x - c), ax = A x
        for (int p0 = 0; p0 < P; p0 += kPC) {
            const int pc = min(kPC, P - p0);
            reduce_chunk<PCMAX>(c, p0, pc, c.I.x, (const double*)nullptr, c.I.x, (const double*)nullptr, true);
            team_reduce<false>(cl, c.vpart, c.vout, pc * Lr, G, g);
            for (int e = c.tid; e < pc * m; e += kThreads) c.ax[p0 * m + e] = c.vout[(e / m) * Lr + e % m];
            for (int e = c.tid; e < pc * k; e += kThreads)
                c.u[p0 * k + e] = c.vout[(e / k) * Lr + 2 * m + e % k];
            __syncthreads();
        }
        double aTwT = 0;
        {
            double acc[1] = {0};
            if (c.I.multi)
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) acc[0] += c.I.alphaT[i] * c.I.cen[i];
            block_reduce<1>(acc, c.spart, c.wred, c.lane, c.warp);
            team_reduce<false>(cl, c.spart, c.sout, 1, G, g);
            aTwT = c.sout[0];
        }
        if constexpr (kIncr) {
            // from here on x, x0, y_D and y_D0 hold double-float pairs
            for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                for (int p = 0; p < P; ++p) {
                    const size_t o = (size_t)p * np + i;
                    const float2 xv = df_split(c.I.x[o]);
                    ((float2*)c.I.x)[o] = xv;
                    ((float2*)c.I.x0)[o] = xv;
                }
                for (int r = 0; r < R; ++r) {
                    const size_t o = (size_t)r * np + i;
                    const float2 yv = df_split(c.I.yD[o]);
                    ((float2*)c.I.yD)[o] = yv;
                    ((float2*)c.I.yD0)[o] = yv;
                }
            }
            asm volatile("fence.proxy.async.global;" ::: "memory");
            __syncthreads();
        }

        lap(0);
        // ---- main loop ---------------------------------------------------------
        long long it = 0;
        int j = 0, restarts = 0;
        int status = FF_MAX_ITER;
        double r_restart = -1, r_prev = INFINITY, r_last = 0;
        double stall_ref = INFINITY;   // relative KKT when it last halved
        int stall_n = 0;               // checks since then
        double res_rel = INFINITY, res_p = 0, res_d = 0, res_g = 0, res_P = 0, res_D = 0, res_T = 0;
        for (it = 0; it < prm.max_iter; ++it) {
            const bool check = (it % prm.check_every) == 0;
            const double cj = (double)(j + 1) / (double)(j + 2);
            const double oj = 1.0 - cj;
            // Halpern step z+ = hlA T(z) + hlB z + hlC z_anchor
            const double hlA = cj * (1.0 + rho), hlB = -cj * rho, hlC = oj;
            // (1) om = Omega u
            apply_omega_m(c, c.u, c.om, P);
            // (2) expand: v = x - tau (grad f(x) + K^T y)
            if constexpr (PCMAX == 1) {
                expand_main_single(c, tau, kap, c.om, c.yAm);
            } else if constexpr (kIncr) {
                // FP32 step u = -tau (grad f + K^T y) and v = x + u, stored as a pair
                // x in FP32 is the second member of the pair buffer (x+ of the last
                // elementwise pass), y_D in FP32 is its FP32 copy: no conversions
                const float* yDf = c.I.yDf;
                float2* v2 = (float2*)c.I.v;
                const float kapf = (float)kap, tauf = (float)tau;
                expand_pass<M, PCMAX>(c, P, c.om, c.yAm, [&](int i, int p, auto aF, auto aA) {
                    const size_t o = (size_t)p * np + i;
                    const float xf = v2[o].y;
                    const float gf = -(float)c.I.alpha[o] +
                                     2.f * kapf * ((float)aF + (float)c.I.Dp[o] * (xf - c.I.cenf[i]));
                    const float kt = (float)aA + yDf[o] - ((p + 1 < R) ? yDf[o + np] : 0.f);
                    const float u = -tauf * (gf + kt);
                    v2[o] = make_float2(xf + u, u);
                });
            } else {
                const double* x = c.I.x;
                const double* yD = c.I.yD;
                double* v = c.I.v;
                const M kapm = (M)kap;
                expand_pass<M, PCMAX>(c, P, c.om, c.yAm, [&](int i, int p, auto aF, auto aA) {
                    // gradient and K^T y in M; the state update in FP64
                    const size_t o = (size_t)p * np + i;
                    const double xv = x[o];
                    const M gf = -(M)c.I.alpha[o] + (M)2 * kapm * ((M)aF + (M)c.I.Dp[o] * (M)(xv - c.I.cen[i]));
                    const M kt = (M)aA + (M)yD[o] - ((p + 1 < R) ? (M)yD[o + np] : (M)0);
                    v[o] = xv - tau * (double)(gf + kt);
                });
            }
            __syncthreads();
            lap(1);
            // (3) thresholds of the l1 projection
            if constexpr (kIncr)
                th_rounds += l1_thresholds(cl, c, (const float2*)c.I.v, c.theta, c.thprev);
            else
                th_rounds += l1_thresholds(cl, c, (const double*)c.I.v, c.theta, c.thprev);
            lap(2);
            // (4) elementwise: x_bar, y_D bar, Halpern combination, residual parts
            //     (fused into the reduce pass for a single period)
            double rloc[2] = {0, 0};
            if constexpr (PCMAX != 1 && kIncr) {
                // FP32 increments on the double-float state: with d1 = x_bar - x (from u
                // and theta) and d0 = x0 - x, x+ = x + hlA d1 + hlC d0; the trade residual
                // of row r is (Delta x + b)_r (a double-float difference rounded once) +
                // 2 (d1_r - d1_{r-1}); the dual update y+ = y + hlA (y_bar - y) + hlC (y0 - y).
                // (x_bar, x+) in FP32 replace (v, u) in the pair buffer for the reduce pass.
                // No FP64 instruction outside the KKT checks.
                const float2* __restrict__ x2 = (const float2*)c.I.x;
                const float2* __restrict__ x02 = (const float2*)c.I.x0;
                const float2* __restrict__ yd2 = (const float2*)c.I.yD;
                const float2* __restrict__ yd02 = (const float2*)c.I.yD0;
                float2* __restrict__ xn2 = (float2*)c.I.xn;
                float2* __restrict__ ydn2 = (float2*)c.I.yDn;
                float2* __restrict__ v2 = (float2*)c.I.v;
                const M* __restrict__ c1a = c.I.c1;
                const M* __restrict__ c2a = c.I.c2;
                const float fA = (float)hlA, fC = (float)hlC, fsD = (float)sD, finv = (float)inv_sD;
                // the thresholds in FP32, once per period (not per element)
                __shared__ float thf_s[64];
                for (int r = c.tid; r < P; r += kThreads) thf_s[r] = (float)c.theta[r];
                __syncthreads();
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                    const float2 w0v = c.I.w0f[i];
                    const float2 wtv = c.I.multi ? c.I.cen2[i] : make_float2(0.f, 0.f);
                    float2 x_prev = make_float2(-w0v.x, -w0v.y);   // row 0 takes b_1 = -w0
                    float d1_prev = 0.f;
                    for (int r = 0; r < R; ++r) {
                        const size_t orr = (size_t)r * np + i;
                        // every load of this row first: none depends on the stores below
                        const float2 yd = yd2[orr];
                        const float2 yd0 = yd02[orr];
                        const float c1v = (float)c1a[orr], c2v = (float)c2a[orr];
                        float2 vu = make_float2(0.f, 0.f), xc = make_float2(0.f, 0.f), x0c = make_float2(0.f, 0.f);
                        if (r < P) {
                            vu = v2[orr];
                            xc = x2[orr];
                            x0c = x02[orr];
                        }
                        float d1 = 0.f;
                        if (r < P) {
                            const float th = thf_s[r];
                            const float av = fabsf(vu.x) - th;
                            float xbf = 0.f;
                            if (av > 0.f) {
                                d1 = vu.y - (vu.x < 0.f ? -th : th);
                                xbf = vu.x < 0.f ? -av : av;
                            } else {
                                d1 = -(xc.x + xc.y);
                            }
                            const float2 xn = df_inc(xc, fA * d1 + fC * df_sub(x0c, xc));
                            xn2[orr] = xn;
                            v2[orr] = make_float2(xbf, xn.x);
                            if (check) {
                                c.I.xb[orr] = av > 0.f ? df_value(xc) + (double)d1 : 0.0;   // exact zeros off the support
                                rloc[0] += (double)d1 * (double)d1;
                            }
                        }
                        // (Delta x + b)_r: x_r - x_{r-1} (x_0 := -b_1 = w0 handled by x_prev),
                        // the last multi-period row adds w_T: then the FP32 correction
                        const float2 cur = (r < P) ? xc : ((c.I.multi && r == R - 1) ? wtv : make_float2(0.f, 0.f));
                        const float dxb = (r == 0 ? (cur.x + x_prev.x) + (cur.y + x_prev.y) : df_sub(cur, x_prev));
                        const float zz = dxb + 2.f * (d1 - d1_prev);
                        x_prev = xc;
                        d1_prev = d1;
                        const float tf = yd.x * finv + zz;
                        float yl, dy;
                        if (trade_multiplier_f(tf, finv, c1v, c2v, dexp, yl)) dy = (yl - yd.x) - yd.y;
                        else dy = fsD * zz;
                        const float2 ydn = df_inc(yd, fA * dy + fC * df_sub(yd0, yd));
                        ydn2[orr] = ydn;
                        c.I.yDf[orr] = ydn.x;
                        if (check) {
                            c.I.yDb[orr] = df_value(yd) + (double)dy;
                            rloc[1] += (double)dy * (double)dy;
                        }
                    }
                }
            } else if constexpr (PCMAX != 1) {
                const double* x = c.I.x;
                const double* v = c.I.v;
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                    double xe_prev = 0;
                    const double w0 = c.I.w0[i];
                    const double wt = c.I.multi ? c.I.cen[i] : 0.0;
                    for (int r = 0; r < R; ++r) {
                        double xe = 0;
                        if (r < P) {
                            const size_t o = (size_t)r * np + i;
                            const double vv = v[o];
                            const double av = fabs(vv) - c.theta[r];
                            const double xb = av > 0 ? (vv < 0 ? -av : av) : 0.0;
                            const double xc = x[o];
                            c.I.xb[o] = xb;
                            xe = 2.0 * xb - xc;
                            c.I.xn[o] = hlA * xb + hlB * xc + hlC * c.I.x0[o];
                            if (check) rloc[0] += (xc - xb) * (xc - xb);
                        }
                        const double dxe = xe - xe_prev;   // (Delta xe)_r; last multi row: -xe_{P-1}
                        xe_prev = xe;
                        const double b = (r == 0 ? -w0 : 0.0) + ((c.I.multi && r == R - 1) ? wt : 0.0);
                        const size_t orr = (size_t)r * np + i;
                        const double yd = c.I.yD[orr];
                        const double pD = yd + sD * dxe;
                        const double t = pD * inv_sD + b;
                        M ylive;
                        const double ydb = trade_multiplier<M>(t, inv_sD, c.I.c1[orr], c.I.c2[orr], dexp, ylive)
                                               ? (double)ylive
                                               : pD + sD * b;
                        c.I.yDb[orr] = ydb;
                        c.I.yDn[orr] = hlA * ydb + hlB * yd + hlC * c.I.yD0[orr];
                        if (check) rloc[1] += (yd - ydb) * (yd - ydb);
                    }
                }
            }
            __syncthreads();
            lap(3);
            // (5) reduce per chunk of periods: A x_bar, A x_new, F^T(x_new - c) [, F^T(x_bar - c)];
            //     then the replicated y_A update and Halpern on y_A
            double rA = 0, pin = 0, nAx = 0, nCl = 0;
            for (int p0 = 0; p0 < P; p0 += kPC) {
                const int pc = min(kPC, P - p0);
                if constexpr (PCMAX == 1)
                    reduce_fused_single(c, hlA, hlB, hlC, sD, inv_sD, dexp, check, rloc);
                else if constexpr (kIncr)
                    reduce_chunk_pairs(c, p0, pc, (const float2*)c.I.v);
                else
                    reduce_chunk<PCMAX>(c, p0, pc, c.I.xb, c.I.xn, c.I.xn, (const double*)nullptr, true);
                team_reduce<false>(cl, c.vpart, c.vout, pc * Lr, G, g);
                for (int e = c.tid; e < pc * m; e += kThreads) {
                    const int q = e / m, jj = e % m;
                    const int pe = (p0 + q) * m + jj;
                    const double abv = c.vout[q * Lr + jj];
                    const double anv = c.vout[q * Lr + m + jj];
                    const double ya = c.yA[pe];
                    const double pA = ya + sA * (2.0 * abv - c.ax[pe]);
                    const double qq = pA * inv_sA;
                    const double cl_ = qq > c.ubd[jj] ? c.ubd[jj] : (qq < c.lb[jj] ? c.lb[jj] : qq);
                    const double yab = pA - sA * cl_;
                    const double yan = hlA * yab + hlB * ya + hlC * c.I.yA0[pe];
                    c.yAb[pe] = yab;
                    c.yA[pe] = yan;
                    c.yAm[pe] = (M)yan;
                    c.ax[pe] = anv;
                    if (check) {
                        rA += (ya - yab) * (ya - yab);
                        const double cla = fmin(fmax(abv, c.lb[jj]), c.ubd[jj]);
                        pin += (abv - cla) * (abv - cla);
                        nAx += abv * abv;
                        nCl += cla * cla;
                    }
                }
                for (int e = c.tid; e < pc * k; e += kThreads) {
                    const int q = e / k, jj = e % k;
                    c.u[(p0 + q) * k + jj] = c.vout[q * Lr + 2 * m + jj];
                }
                __syncthreads();
                if (check) {
                    // F^T (x_bar - c) for the KKT check in FP64 products: the objective
                    // term kappa u^T Omega u must not carry the FP32 product error.
                    // Sub-chunks of <= 4 periods; their count depends on pc only, so
                    // every CTA of the cluster takes the same team reductions
                    for (int s0 = 0; s0 < pc; s0 += 4) {
                        const int sc = min(4, pc - s0);
                        reduce_chunk_f64<PCMAX>(c, p0 + s0, sc, c.I.xb);
                        team_reduce<false>(cl, c.vpart, c.vout, sc * Lr, G, g);
                        for (int e = c.tid; e < sc * k; e += kThreads) {
                            const int q = e / k, jj = e % k;
                            c.ub[(p0 + s0 + q) * k + jj] = c.vout[q * Lr + 2 * m + k + jj];
                        }
                        __syncthreads();
                    }
                }
            }
            // rotate iterate buffers: x <- x_new, y_D <- y_D new
            {
                double* t1 = c.I.x; c.I.x = c.I.xn; c.I.xn = t1;
                double* t2 = c.I.yD; c.I.yD = c.I.yDn; c.I.yDn = t2;
            }
            ++j;
            lap(4);
            if (!check) continue;

            // ---- (6) check: fixed-point residual and relative KKT at T(z), FP64 ----
            // q = x_bar - (grad f + K^T y) needs a P x np FP64 buffer: v, except in the
            // multi-period FP32-increment iteration, whose pair buffer must survive
            // (it carries x in FP32): there the retired iterate buffer x+ serves
            double* qbuf = (kIncr && PCMAX != 1) ? c.I.xn : c.I.v;
            // replicated parts (every CTA holds them): factor term of f at x_bar
            double fF = 0;
            for (int e = c.tid; e < P * k; e += kThreads) {
                const int p = e / k, jj = e % k;
                double s;
                if (c.I.omega_diag) {
                    s = c.Om[jj] * c.ub[e];
                } else {
                    s = 0;
                    for (int l = 0; l < k; ++l) s += c.Om[jj * k + l] * c.ub[p * k + l];
                }
                fF += c.ub[e] * s;
            }
            double rep[5] = {rA, pin, nAx, nCl, fF};
            block_reduce<5>(rep, c.spart + 32, c.wred, c.lane, c.warp);
            const double rA_t = c.spart[32], pin_t = c.spart[33], nAx_t = c.spart[34], nCl_t = c.spart[35];
            const double fF_t = c.spart[36];
            __syncthreads();
            // Omega u_bar in place for the gradient at x_bar
            if (c.I.omega_diag) {
                for (int e = c.tid; e < P * k; e += kThreads) c.ub[e] *= c.Om[e % k];
                __syncthreads();
            } else {
                for (int p = 0; p < P; ++p) {
                    for (int jj = c.tid; jj < k; jj += kThreads) {
                        double s = 0;
                        for (int l = 0; l < k; ++l) s += c.Om[jj * k + l] * c.ub[p * k + l];
                        c.vout[jj] = s;
                    }
                    __syncthreads();
                    for (int jj = c.tid; jj < k; jj += kThreads) c.ub[p * k + jj] = c.vout[jj];
                    __syncthreads();
                }
            }
            double kloc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            {
                const double* xb = c.I.xb;
                const double* ydb = c.I.yDb;
                double* qv = qbuf;
                expand_pass<double, PCMAX>(c, P, c.ub, c.yAb, [&](int i, int p, auto aF, auto aA) {
                    const size_t o = (size_t)p * np + i;
                    const double xv = xb[o];
                    const double dx = xv - c.I.cen[i];
                    const double gf = -c.I.alpha[o] + 2.0 * kap * (aF + c.I.Dp[o] * dx);
                    const double kt = aA + ydb[o] - ((p + 1 < R) ? ydb[o + np] : 0.0);
                    qv[o] = xv - (gf + kt);
                    kloc[0] += -c.I.alpha[o] * xv + kap * c.I.Dp[o] * dx * dx;   // f without factor term
                    kloc[1] += gf * xv;                                          // <grad f, x>
                    kloc[2] += xv * xv;
                    kloc[3] += gf * gf;
                    kloc[4] += kt * kt;
                    kloc[7] += kap * c.I.Dp[o] * dx * dx;                        // specific risk
                    kloc[8] += fabs(c.I.alpha[o] * xv);                          // return magnitudes
                });
                // trade costs phi(Delta x_bar + b) and h_D*(yD_bar) = -<y, b> + sum phi*(y)
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                    double prevx = 0;
                    const double w0 = c.I.w0[i];
                    const double wt = c.I.multi ? c.I.cen[i] : 0.0;
                    for (int r = 0; r < R; ++r) {
                        const double xv = (r < P) ? xb[(size_t)r * np + i] : 0.0;
                        const double b = (r == 0 ? -w0 : 0.0) + ((c.I.multi && r == R - 1) ? wt : 0.0);
                        const double z = xv - prevx + b;
                        prevx = xv;
                        const size_t orr = (size_t)r * np + i;
                        const double c1 = c.I.c1[orr], c2 = c.I.c2[orr];
                        const double az = fabs(z);
                        kloc[5] += c1 * az + c2 * pow(az, dexp);
                        const double y = ydb[orr];
                        kloc[6] += -y * b + cost_conj(y, c1, c2, dexp);
                    }
                }
            }
            double part[11] = {rloc[0], rloc[1], kloc[0], kloc[1], kloc[2], kloc[3],
                               kloc[4], kloc[5], kloc[6], kloc[7], kloc[8]};
            block_reduce<11>(part, c.spart, c.wred, c.lane, c.warp);
            if (c.tid == 0) {
                c.spart[11] = (g == 0) ? (double)(globaltimer() - t_start) : 0.0;
                c.spart[12] = (double)pipe_err_s;
            }
            __syncthreads();
            team_reduce<false>(cl, c.spart, c.sout, 13, G, g);
            double sums[13];
            for (int e = 0; e < 13; ++e) sums[e] = c.sout[e];
            __syncthreads();
            // per-period max_i |grad f + K^T y| = |x_bar - q|   (g*(-grad f - K^T y))
            for (int p = 0; p < P; ++p) {
                double mx[1] = {0};
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                    const size_t o = (size_t)p * np + i;
                    mx[0] = fmax(mx[0], fabs(c.I.xb[o] - qbuf[o]));
                }
                block_reduce<1, true>(mx, c.spart + p, c.wred, c.lane, c.warp);
            }
            team_reduce<true>(cl, c.spart, c.sout, P, G, g);
            double gstar = 0;
            for (int p = 0; p < P; ++p) gstar += c.sout[p];
            __syncthreads();
            // stationarity residual ||x_bar - Proj(q)||  (thresholds warm-started
            // from the previous check)
            l1_thresholds(cl, c, (const double*)qbuf, c.theta, c.thq);
            double dr[1] = {0};
            for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                for (int p = 0; p < P; ++p) {
                    const size_t o = (size_t)p * np + i;
                    const double qv = qbuf[o];
                    const double aq = fabs(qv) - c.theta[p];
                    const double pq = aq > 0 ? (qv < 0 ? -aq : aq) : 0.0;
                    const double dd = c.I.xb[o] - pq;
                    dr[0] += dd * dd;
                }
            }
            block_reduce<1>(dr, c.spart, c.wred, c.lane, c.warp);
            team_reduce<false>(cl, c.spart, c.sout, 1, G, g);
            const double rd_num = sqrt(c.sout[0]);
            __syncthreads();
            double hA = 0;
            for (int e = 0; e < P * m; ++e) {
                const int jj = e % m;
                const double y = c.yAb[e];
                if (y > 0) hA += y * c.ubd[jj];
                else if (y < 0) hA += y * c.lb[jj];
            }
            const double fval = sums[2] + kap * fF_t;
            const double Pobj = fval + sums[7];
            const double Dobj = fval - sums[3] - gstar - hA - sums[8];
            const double r_p = sqrt(pin_t) / (sqrt(nAx_t) + sqrt(nCl_t) + 1e-30);
            const double r_d = rd_num / (sqrt(sums[4]) + sqrt(sums[5]) + sqrt(sums[6]) + 1e-30);
            // purely relative gap |P - D| / (|P| + |D|); the magnitude of the
            // objective's terms (return magnitudes + risk + trading cost) is
            // reported beside it (ff_result.term_scale)
            const double phi_terms = sums[10] + sums[9] + kap * fF_t + sums[7];
            const double r_g = fabs(Pobj - Dobj) / (fabs(Pobj) + fabs(Dobj) + 1e-30);
            const double rel = fmax(r_p, fmax(r_d, r_g));
            const double fpr = sqrt(sums[0] / tau + sums[1] / sD + rA_t / sA);
            res_rel = rel; res_p = r_p; res_d = r_d; res_g = r_g; res_P = Pobj; res_D = Dobj; res_T = phi_terms;
            r_last = fpr;
            lap(5);
            int st_new = -1;   // a stop status, or -1 to go on
            if (sums[12] > 0) {
                st_new = FF_STALLED;
            } else if (!(r_p == r_p) || !(r_d == r_d) || !(r_g == r_g) || !(fpr == fpr) || !(Pobj == Pobj) ||
                       !(Dobj == Dobj) || isinf(Pobj) || isinf(Dobj)) {
                // every part is tested: fmax would pass over a NaN in one of them
                st_new = FF_NUMERICAL;
            } else if (rel <= prm.tol) {
                st_new = FF_CONVERGED;
            } else if (sums[11] > prm.time_limit_ns) {
                st_new = FF_TIME_LIMIT;
            } else {
                // precision floor of the FP32/BF16 modes: no halving of the relative
                // KKT residual over stall_checks checks (the rounding of the FP32
                // products then bounds it; the host re-solves such instances in FP64)
                if (rel <= 0.5 * stall_ref) { stall_ref = rel; stall_n = 0; }
                else ++stall_n;
                if (kIncr && prm.stall_checks > 0 && stall_n >= prm.stall_checks) st_new = FF_PRECISION;
            }
            bool do_restart = false;
            if (st_new < 0) {
                // restart on the fixed-point residual: sufficient decay, necessary
                // decay that stalls, or (artificial) once the current restart cycle
                // holds a fixed share of all iterations so far; the anchor becomes
                // the current iterate
                if (r_restart < 0) r_restart = fpr;
                do_restart = (fpr <= prm.beta_suff * r_restart) ||
                             (fpr <= prm.beta_nec * r_restart && fpr > r_prev) ||
                             (prm.beta_art > 0 && (double)j >= prm.beta_art * (double)(it + 1));
                r_prev = fpr;
            }
            // every CTA of the team takes rank 0's decisions (they are computed from
            // bit-identical team sums; the broadcast keeps the team's control flow,
            // and so its cluster barriers, uniform by construction)
            if (g == 0 && c.tid == 0) {
                decide_s[0] = st_new;
                decide_s[1] = do_restart ? 1 : 0;
            }
            cl.sync();
            {
                const int* d0 = cl.map_shared_rank(decide_s, 0);
                st_new = d0[0];
                do_restart = d0[1] != 0;
            }
            cl.sync();
            if (st_new >= 0) {
                if (st_new == FF_NUMERICAL) res_rel = NAN;
                status = st_new;
                break;
            }
            if (do_restart) {
                // distances travelled since the last restart (primal weight), then
                // the current iterate becomes the anchor
                double dl[3] = {0.0, 0.0, 0.0};
                for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
                    for (int p = 0; p < P; ++p) {
                        const size_t o = (size_t)p * np + i;
                        double dd;
                        if constexpr (kIncr) dd = (double)df_sub(((const float2*)c.I.x)[o], ((const float2*)c.I.x0)[o]);
                        else dd = c.I.x[o] - c.I.x0[o];
                        dl[0] += dd * dd;
                        c.I.x0[o] = c.I.x[o];
                    }
                    for (int r = 0; r < R; ++r) {
                        const size_t o = (size_t)r * np + i;
                        double dd;
                        if constexpr (kIncr) dd = (double)df_sub(((const float2*)c.I.yD)[o], ((const float2*)c.I.yD0)[o]);
                        else dd = c.I.yD[o] - c.I.yD0[o];
                        dl[1] += dd * dd;
                        c.I.yD0[o] = c.I.yD[o];
                    }
                }
                // y_A and its anchor are replicated in every CTA of the team (the
                // anchor in one global array that every CTA writes with the same
                // values): rank 0 alone counts their distance, and no CTA writes the
                // new anchor before the team reduction below, whose cluster barriers
                // order every CTA's reads of the old anchor before those writes; so
                // every CTA holds bit-identical distances and takes the same decisions
                if (g == 0)
                    for (int e = c.tid; e < P * m; e += kThreads) {
                        const double dd = c.yA[e] - c.I.yA0[e];
                        dl[2] += dd * dd;
                    }
                block_reduce<3>(dl, c.spart, c.wred, c.lane, c.warp);
                team_reduce<false>(cl, c.spart, c.sout, 3, G, g);
                const double dx = sqrt(c.sout[0]), dy = sqrt(c.sout[1] + c.sout[2]);
                for (int e = c.tid; e < P * m; e += kThreads) c.I.yA0[e] = c.yA[e];
                // the new anchor is read by bulk copies (async proxy) from here on
                asm volatile("fence.proxy.async.global;" ::: "memory");
                __syncthreads();
                j = 0;
                ++restarts;
                r_restart = fpr;
                r_prev = INFINITY;
                if (prm.primal_weight && dx > 1e-30 && dy > 1e-30) {
                    const double target = fmin(fmax(dy / dx, 1e-4 * omega0), 1e4 * omega0);
                    omega = exp(0.5 * log(target) + 0.5 * log(omega));
                    set_steps(omega);
                    r_restart = -1.0;   // the next check measures in the new step metric
                }
            }
        }

        // a frozen ring may still have copies landing in its stages: let them
        // land before the outputs and the next instance (bounded waits)
        __syncthreads();
        if (c.pipe.frozen && !ring_broken_s) {
            const bool ok = pipe_drain(c.pipe);
            if (!ok && threadIdx.x == 0) ring_broken_s = 1;
            if (!ok) c.pipe.frozen = 1;
        }
        // ---- outputs: T(z) of the last check (x_bar, y_bar) -----------------
        __syncthreads();
        for (int i = c.i0 + c.tid; i < c.i1; i += kThreads) {
            for (int p = 0; p < P; ++p) {
                const double val = c.I.xb[(size_t)p * np + i];
                if (c.I.out_f64) ((double*)c.I.w_out)[(size_t)p * n + i] = val;
                else ((float*)c.I.w_out)[(size_t)p * n + i] = (float)val;
            }
            if (c.I.yD_out) {
                for (int r = 0; r < R; ++r) {
                    const double val = c.I.yDb[(size_t)r * np + i];
                    if (c.I.out_f64) ((double*)c.I.yD_out)[(size_t)r * n + i] = val;
                    else ((float*)c.I.yD_out)[(size_t)r * n + i] = (float)val;
                }
            }
        }
        if (g == 0 && c.I.yA_out) {
            for (int e = c.tid; e < P * m; e += kThreads) {
                const double val = c.yAb[e];
                if (c.I.out_f64) ((double*)c.I.yA_out)[e] = val;
                else ((float*)c.I.yA_out)[e] = (float)val;
            }
        }
        if (g == 0 && c.tid == 0) {
            ff_result rs;
            rs.status = status;
            rs.restarts = restarts;
            rs.iterations = (int64_t)(status == FF_MAX_ITER ? it : it + 1);
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
            rs.threshold_rounds = th_rounds;
            for (int q = 0; q < 6; ++q) rs.phase_seconds[q] = ph[q] * 1e-9;
            rs.term_scale = res_T;
            *c.I.res = rs;
        }
        pipe = c.pipe;
        // the next instance reuses shared memory: every rank must be done with it
        cl.sync();
    }
    // every instance drained its ring before the team moved on; only a copy
    // that never landed (ring_broken_s, a hardware fault) can still be pending
}

template <class M, class S, int PCMAX>
static cudaError_t prepare(int G, size_t smem) {
    auto kern = team_kernel<M, S, PCMAX>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (G > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

static cudaLaunchConfig_t team_config(int G, int nteams, size_t smem, cudaStream_t stream, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(G * nteams), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <class M, class S>
cudaError_t launch_solver(const Inst<M, S>* insts, int count, const Params& prm, int G, int nteams, size_t smem,
                          bool single, cudaStream_t stream) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = team_config(G, nteams, smem, stream, attr);
    if (single) {
        cudaError_t e = prepare<M, S, 1>(G, smem);
        if (e != cudaSuccess) return e;
        return cudaLaunchKernelEx(&cfg, team_kernel<M, S, 1>, insts, count, prm);
    }
    cudaError_t e = prepare<M, S, kPC>(G, smem);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, team_kernel<M, S, kPC>, insts, count, prm);
}

template <class M, class S>
cudaError_t max_teams(int G, size_t smem, bool single, int* out) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = team_config(G, 1, smem, 0, attr);
    if (single) {
        cudaError_t e = prepare<M, S, 1>(G, smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveClusters(out, team_kernel<M, S, 1>, &cfg);
    }
    cudaError_t e = prepare<M, S, kPC>(G, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveClusters(out, team_kernel<M, S, kPC>, &cfg);
}

template cudaError_t launch_solver<double, double>(const Inst<double, double>*, int, const Params&, int, int,
                                                   size_t, bool, cudaStream_t);
template cudaError_t launch_solver<float, float>(const Inst<float, float>*, int, const Params&, int, int, size_t,
                                                 bool, cudaStream_t);
template cudaError_t launch_solver<float, __nv_bfloat16>(const Inst<float, __nv_bfloat16>*, int, const Params&,
                                                         int, int, size_t, bool, cudaStream_t);
template cudaError_t max_teams<double, double>(int, size_t, bool, int*);
template cudaError_t max_teams<float, float>(int, size_t, bool, int*);
template cudaError_t max_teams<float, __nv_bfloat16>(int, size_t, bool, int*);

}  // namespace ff
