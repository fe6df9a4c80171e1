// ks_hmmw.cuh -- the discrete-state (HMM) filter and smoother for K = 16 and
// 32 states: one K-lane group of a warp per chain of steps, lane z holding
// row z of each K x K element (Section III's Definitions 1 and 2 with sums,
// as in ks_hmm.cuh).
//
// A chain's elements are too large for one thread's registers at this K, so
// every scan runs as reduce / spine / apply launches (as the nx = 8 and
// nx = 32 Gaussian paths do):
//  * forward reduce: each warp folds its chain's step elements into one
//    Definition 1 element; warp 0 combines the block's chains in order,
//    storing each chain's exclusive in-tile prefix and the tile aggregate;
//  * spine: Kogge-Stone over the tile aggregates (one launch per level);
//  * forward apply: each chain starts from its prefix (all rows equal:
//    p(x | y_1:k) and log p(y_1:k)), steps through its measurements writing
//    filt and loglik, and folds its Definition 2 elements into one chain
//    smoothing aggregate;
//  * reverse reduce / spine / apply over those aggregates in reversed order,
//    the apply walking each chain backwards from its suffix.
// Likelihood rows are scaled to a maximum of 1 and g is kept as log g, so
// that p(y_1:k) survives long prefixes in FP32; products of row-stochastic
// matrices are rescaled to unit row sums.
#pragma once

#include "ks_scan.cuh"

namespace ks {
namespace hmmw {

// Shared-memory pitches: Pi rows are read by all lanes of a chain at once
// (broadcast) or a column per lane, so pitch K with float4 rows; Pi^T is read a
// row per lane, so an odd pitch; element slots are written a row per lane with
// float4 stores and read by broadcast, so pitch Q (a multiple of 4, rows in
// distinct banks per quarter-warp).
template <int K>
struct Dims {
    static constexpr int PT = K + 1;
    static constexpr int Q = K + 4;
    static constexpr int SLOT = K * Q + K;       // rows, then log g
    static constexpr int FREC = K * K + K;       // global filtering record: rows, then log g
    static constexpr int SREC = K * K;           // global smoothing record: rows
};

// A chain is K lanes of one warp (lane z = row z); 32 / K chains per warp.
template <int K>
KS_DEV unsigned gmask() {
    if constexpr (K == 32) return 0xffffffffu;
    else return ((1u << K) - 1u) << (threadIdx.x & (32 - K));
}

template <int K>
KS_DEV int glane() { return threadIdx.x & (K - 1); }

template <int K>
struct Const {
    float Pi[K * K];
    float q1[K];   // p(x_1) = pi Pi
};

// One warp's share of a filtering element: lane z holds row z and lg[z].
template <int K>
struct FRow {
    float f[K];
    float lg;
};

template <int K>
KS_DEV float group_sum(float v) {
#pragma unroll
    for (int o = K / 2; o > 0; o >>= 1) v += __shfl_xor_sync(gmask<K>(), v, o, K);
    return v;
}

// Pi (pitch K) and its transpose (pitch PT) into shared memory.
template <int K>
KS_DEV void load_pi(const Const<K>* __restrict__ cg, float* __restrict__ Pi, float* __restrict__ PiT, float* q1) {
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const float v = __ldg(cg->Pi + e);
        Pi[e] = v;
        PiT[(e % K) * Dims<K>::PT + e / K] = v;
    }
    for (int e = threadIdx.x; e < K; e += blockDim.x) q1[e] = __ldg(cg->q1 + e);
}

template <int K>
KS_DEV void load_frow(const float* __restrict__ src, FRow<K>& r) {
    const int z = glane<K>();
    const float4* p = reinterpret_cast<const float4*>(src + z * K);
#pragma unroll
    for (int i = 0; i < K / 4; ++i) {
        const float4 q = __ldcg(p + i);
        r.f[4 * i] = q.x;
        r.f[4 * i + 1] = q.y;
        r.f[4 * i + 2] = q.z;
        r.f[4 * i + 3] = q.w;
    }
    r.lg = __ldcg(src + K * K + z);
}

template <int K>
KS_DEV void store_frow(float* __restrict__ dst, const FRow<K>& r) {
    const int z = glane<K>();
    float4* p = reinterpret_cast<float4*>(dst + z * K);
#pragma unroll
    for (int i = 0; i < K / 4; ++i) p[i] = make_float4(r.f[4 * i], r.f[4 * i + 1], r.f[4 * i + 2], r.f[4 * i + 3]);
    dst[K * K + z] = r.lg;
}

template <int K>
KS_DEV void load_srow(const float* __restrict__ src, float (&a)[K]) {
    const float4* p = reinterpret_cast<const float4*>(src + glane<K>() * K);
#pragma unroll
    for (int i = 0; i < K / 4; ++i) {
        const float4 q = __ldcg(p + i);
        a[4 * i] = q.x;
        a[4 * i + 1] = q.y;
        a[4 * i + 2] = q.z;
        a[4 * i + 3] = q.w;
    }
}

template <int K>
KS_DEV void store_srow(float* __restrict__ dst, const float (&a)[K]) {
    float4* p = reinterpret_cast<float4*>(dst + glane<K>() * K);
#pragma unroll
    for (int i = 0; i < K / 4; ++i) p[i] = make_float4(a[4 * i], a[4 * i + 1], a[4 * i + 2], a[4 * i + 3]);
}

// A chain's element in a shared-memory slot (pitch Q rows, then lg).
template <int K>
KS_DEV void put_srow(float* __restrict__ buf, const float (&a)[K]) {
    float4* p = reinterpret_cast<float4*>(buf + glane<K>() * Dims<K>::Q);
#pragma unroll
    for (int i = 0; i < K / 4; ++i) p[i] = make_float4(a[4 * i], a[4 * i + 1], a[4 * i + 2], a[4 * i + 3]);
}

template <int K>
KS_DEV void put_frow(float* __restrict__ buf, const FRow<K>& r) {
    put_srow(buf, r.f);
    buf[K * Dims<K>::Q + glane<K>()] = r.lg;
}

// Row y of a K x K shared-memory matrix with a 16-byte-aligned pitch, as float4s.
template <int PITCH, int K>
KS_DEV void smem_row(const float* __restrict__ M, int y, float (&v)[K]) {
    const float4* p = reinterpret_cast<const float4*>(M + y * PITCH);
#pragma unroll
    for (int i = 0; i < K / 4; ++i) {
        const float4 q = p[i];
        v[4 * i] = q.x;
        v[4 * i + 1] = q.y;
        v[4 * i + 2] = q.z;
        v[4 * i + 3] = q.w;
    }
}

// Likelihood row of step k, the same for every lane, scaled to a maximum of
// 1; returns the log of the maximum.
template <int K>
KS_DEV float lik_row(const float* __restrict__ lik, int64_t k, float (&l)[K], Flags& bad) {
    const float4* p = reinterpret_cast<const float4*>(lik + k * K);
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < K / 4; ++i) {
        const float4 q = __ldg(p + i);
        l[4 * i] = q.x;
        l[4 * i + 1] = q.y;
        l[4 * i + 2] = q.z;
        l[4 * i + 3] = q.w;
    }
#pragma unroll
    for (int x = 0; x < K; ++x) m = fmaxf(m, l[x]);
    bad |= !(m > 0.f) || !(m <= 3.0e38f);
    const float r = 1.f / m;
#pragma unroll
    for (int x = 0; x < K; ++x) l[x] *= r;
    return __logf(m);
}

// Row z of the step element: Pi[z][x] l(x) normalised, lg = lm + log(row sum).
template <int K>
KS_DEV void step_row(FRow<K>& r, const float* __restrict__ Pi, const float (&l)[K], float lm, Flags& bad) {
    const int z = glane<K>();
    float s = 0.f;
    smem_row<K>(Pi, z, r.f);
#pragma unroll
    for (int x = 0; x < K; ++x) {
        r.f[x] *= l[x];
        s += r.f[x];
    }
    bad |= !(s > 0.f);
    const float rs = 1.f / s;
#pragma unroll
    for (int x = 0; x < K; ++x) r.f[x] *= rs;
    r.lg = lm + __logf(s);
}

// The k = 1 element: every row p(x_1 | y_1), lg = log p(y_1).
template <int K>
KS_DEV void first_row(FRow<K>& r, const float* __restrict__ q1, const float (&l)[K], float lm, Flags& bad) {
    float s = 0.f;
#pragma unroll
    for (int x = 0; x < K; ++x) {
        r.f[x] = q1[x] * l[x];
        s += r.f[x];
    }
    bad |= !(s > 0.f);
    const float rs = 1.f / s;
#pragma unroll
    for (int x = 0; x < K; ++x) r.f[x] *= rs;
    r.lg = lm + __logf(s);
}

// Fold of a step element into row z: (f Pi)[z] . l, normalised.
template <int K>
KS_DEV void fold_row(FRow<K>& r, const float* __restrict__ Pi, const float (&l)[K], float lm, Flags& bad) {
    float o[K];
#pragma unroll
    for (int x = 0; x < K; ++x) o[x] = 0.f;
#pragma unroll
    for (int y = 0; y < K; ++y) {
        float pr[K];
        smem_row<K>(Pi, y, pr);
#pragma unroll
        for (int x = 0; x < K; ++x) o[x] = fmaf(r.f[y], pr[x], o[x]);
    }
    float s = 0.f;
#pragma unroll
    for (int x = 0; x < K; ++x) {
        o[x] *= l[x];
        s += o[x];
    }
    bad |= !(s > 0.f);
    const float rs = 1.f / s;
#pragma unroll
    for (int x = 0; x < K; ++x) r.f[x] = o[x] * rs;
    r.lg += lm + __logf(s);
}

// Definition 1, (row z of a_i, in registers) (x) a_j (in shared memory).
template <int K>
KS_DEV void combine_row(FRow<K>& r, const float* __restrict__ ej, Flags& bad) {
    float mx = ej[K * Dims<K>::Q];
#pragma unroll
    for (int y = 1; y < K; ++y) mx = fmaxf(mx, ej[K * Dims<K>::Q + y]);
    float o[K], d = 0.f;
#pragma unroll
    for (int x = 0; x < K; ++x) o[x] = 0.f;
#pragma unroll
    for (int y = 0; y < K; ++y) {
        const float fw = r.f[y] * __expf(ej[K * Dims<K>::Q + y] - mx);
        d += fw;
        float er[K];
        smem_row<Dims<K>::Q>(ej, y, er);
#pragma unroll
        for (int x = 0; x < K; ++x) o[x] = fmaf(fw, er[x], o[x]);
    }
    bad |= !(d > 0.f);
    const float rd = 1.f / d;
#pragma unroll
    for (int x = 0; x < K; ++x) r.f[x] = o[x] * rd;
    r.lg += mx + __logf(d);
}

// Row z of (a in registers) times (b in shared memory), rescaled to sum 1.
template <int K>
KS_DEV void matmul_row(float (&a)[K], const float* __restrict__ b) {
    float o[K];
#pragma unroll
    for (int x = 0; x < K; ++x) o[x] = 0.f;
#pragma unroll
    for (int y = 0; y < K; ++y) {
        float br[K];
        smem_row<Dims<K>::Q>(b, y, br);
#pragma unroll
        for (int x = 0; x < K; ++x) o[x] = fmaf(a[y], br[x], o[x]);
    }
    float s = 0.f;
#pragma unroll
    for (int x = 0; x < K; ++x) s += o[x];
    const float rs = 1.f / s;
#pragma unroll
    for (int x = 0; x < K; ++x) a[x] = o[x] * rs;
}

// The prefix (all rows equal) as a state: lane x takes p(x) from row 0.
template <int K>
KS_DEV void row0_state(const FRow<K>& r, float& p, float& L) {
    const int lane = glane<K>();
    p = 0.f;
#pragma unroll
    for (int x = 0; x < K; ++x) {
        const float v = __shfl_sync(gmask<K>(), r.f[x], 0, K);
        if (lane == x) p = v;
    }
    L = __shfl_sync(gmask<K>(), r.lg, 0, K);
}

template <int K>
KS_DEV float row0_vec(const float (&a)[K]) {
    const int lane = glane<K>();
    float s = 0.f;
#pragma unroll
    for (int x = 0; x < K; ++x) {
        const float v = __shfl_sync(gmask<K>(), a[x], 0, K);
        if (lane == x) s = v;
    }
    return s;
}

// Filtering state (lane x: p(x)) (x) step: p'(x) = (p Pi)(x) l(x) / c.
template <int K>
KS_DEV void advance_step(float& p, float& L, float& comp, const float* __restrict__ Pi, float lx, float lm,
                         Flags& bad) {
    const int x = glane<K>();
    float o = 0.f;
#pragma unroll
    for (int y = 0; y < K; ++y) o = fmaf(__shfl_sync(gmask<K>(), p, y, K), Pi[y * K + x], o);
    const float v = o * lx;
    const float c = group_sum<K>(v);
    bad |= !(c > 0.f);
    p = v / c;
    const float t = (lm + __logf(c)) - comp;   // Kahan-compensated running log-likelihood
    const float Ln = L + t;
    comp = (Ln - L) - t;
    L = Ln;
}

// Row z of the step's Definition 2 element from its filtered marginal
// (lane x: p(x)): a(x | z) = p(x) Pi[x][z] / sum_x' p(x') Pi[x'][z].
template <int K>
KS_DEV void selem_row(float (&a)[K], float p, const float* __restrict__ PiT, Flags& bad) {
    const int z = glane<K>();
    float d = 0.f;
#pragma unroll
    for (int x = 0; x < K; ++x) {
        a[x] = __shfl_sync(gmask<K>(), p, x, K) * PiT[z * Dims<K>::PT + x];
        d += a[x];
    }
    bad |= !(d > 0.f);
    const float rd = 1.f / d;
#pragma unroll
    for (int x = 0; x < K; ++x) a[x] *= rd;
}

template <int K>
KS_DEV void selem_last_row(float (&a)[K], float p) {
#pragma unroll
    for (int x = 0; x < K; ++x) a[x] = __shfl_sync(gmask<K>(), p, x, K);
}

// Smoothing state (lane x: s(x)) advanced through the step's element built
// from p (lane x: p(x)):  s'(x) = p(x) sum_z (s(z) / d(z)) Pi[x][z],
// d(z) = sum_x p(x) Pi[x][z]; rescaled to sum 1.
template <int K>
KS_DEV void sadvance_step(float& s, float p, const float* __restrict__ PiT, Flags& bad) {
    const int lane = glane<K>();
    float d = 0.f;   // lane z: d(z)
#pragma unroll
    for (int x = 0; x < K; ++x) d = fmaf(__shfl_sync(gmask<K>(), p, x, K), PiT[lane * Dims<K>::PT + x], d);
    bad |= !(d > 0.f);
    const float v = s / d;
    float o = 0.f;   // lane x
#pragma unroll
    for (int z = 0; z < K; ++z) o = fmaf(__shfl_sync(gmask<K>(), v, z, K), PiT[z * Dims<K>::PT + lane], o);
    const float sn = p * o;
    s = sn / group_sum<K>(sn);
}

// ---------------------------------------------------------------- kernels
struct Bufs {
    float* fexcl;     // [nchains][FREC] exclusive in-tile prefixes of the forward scan
    float* fspine0;   // [ntiles][FREC]
    float* fspine1;
    float* schain;    // [nchains][SREC] chain smoothing aggregates (forward apply)
    float* sexcl;     // [nchains][SREC]
    float* sspine0;   // [ntiles][SREC]
    float* sspine1;
};

// NG = NW * 32 / K chains per block (one K-lane group each).
template <int K, int NW>
struct alignas(16) Smem {
    static constexpr int NG = NW * 32 / K;
    float Pi[K * K];
    float PiT[K * Dims<K>::PT];
    float q1[K];
    float pad[(4 - (K * Dims<K>::PT + K) % 4) % 4];
    float slot[NG][Dims<K>::SLOT];   // one element per chain (pitch Q rows + lg)
};

template <int K, int NW, int CH>
__global__ void __launch_bounds__(NW * 32) filter_reduce_kernel(const Const<K>* __restrict__ cg,
                                                                const float* __restrict__ lik, int64_t T, Bufs b,
                                                                uint32_t* status) {
    __shared__ Smem<K, NW> sm;
    constexpr int NG = Smem<K, NW>::NG;
    load_pi(cg, sm.Pi, sm.PiT, sm.q1);
    __syncthreads();
    const int w = threadIdx.x / K;
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t c = (int64_t)blockIdx.x * NG + w;
    const int64_t left = nch - (int64_t)blockIdx.x * NG;
    const int nvalid = left < NG ? (int)left : NG;
    Flags bad = 0u;
    if (w < nvalid) {
        const int64_t k0 = c * CH, k1 = (k0 + CH < T) ? k0 + CH : T;
        FRow<K> r;
        float l[K];
        float lm = lik_row(lik, k0, l, bad);
        if (k0 == 0) first_row(r, sm.q1, l, lm, bad);
        else step_row(r, sm.Pi, l, lm, bad);
#pragma unroll 1
        for (int64_t k = k0 + 1; k < k1; ++k) {
            lm = lik_row(lik, k, l, bad);
            fold_row(r, sm.Pi, l, lm, bad);
        }
        put_frow(sm.slot[w], r);
    }
    __syncthreads();
    if (w == 0) {   // in-tile combine, chain order
        FRow<K> acc;
        smem_row<Dims<K>::Q>(sm.slot[0], glane<K>(), acc.f);
        acc.lg = sm.slot[0][K * Dims<K>::Q + glane<K>()];
#pragma unroll 1
        for (int t = 1; t < nvalid; ++t) {
            store_frow(b.fexcl + ((int64_t)blockIdx.x * NG + t) * Dims<K>::FREC, acc);
            combine_row(acc, sm.slot[t], bad);
        }
        store_frow(b.fspine0 + (int64_t)blockIdx.x * Dims<K>::FREC, acc);
    }
    report_flags(status, bad, kFull, (threadIdx.x & 31) == 0);
}

// Kogge-Stone level s over tile aggregates: dst[t] = src[t - s] (x) src[t].
// FILTER: Definition 1 records; else smoothing records in scan (reversed
// time) order, combined as the matrix product src[t - s] src[t].
template <bool FILTER, int K, int NW>
__global__ void __launch_bounds__(NW * 32) spine_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                        int ntiles, int s, uint32_t* status) {
    constexpr int NG = NW * 32 / K;
    __shared__ __align__(16) float slot[NG][Dims<K>::SLOT];
    constexpr int REC = FILTER ? Dims<K>::FREC : Dims<K>::SREC;
    const int w = threadIdx.x / K;
    const int t = blockIdx.x * NG + w;
    Flags bad = 0u;
    if (t < ntiles) {
        if (t >= s) {
            if constexpr (FILTER) {
                FRow<K> r;
                load_frow(src + (int64_t)t * REC, r);
                put_frow(slot[w], r);
                __syncwarp(gmask<K>());
                load_frow(src + (int64_t)(t - s) * REC, r);
                combine_row(r, slot[w], bad);
                store_frow(dst + (int64_t)t * REC, r);
            } else {
                float a[K];
                load_srow(src + (int64_t)t * REC, a);
                put_srow(slot[w], a);
                __syncwarp(gmask<K>());
                load_srow(src + (int64_t)(t - s) * REC, a);
                matmul_row(a, slot[w]);
                store_srow(dst + (int64_t)t * REC, a);
            }
        } else {
            const float4* p = reinterpret_cast<const float4*>(src + (int64_t)t * REC);
            float4* q = reinterpret_cast<float4*>(dst + (int64_t)t * REC);
            for (int i = glane<K>(); i < REC / 4; i += K) q[i] = __ldcg(p + i);
        }
    }
    report_flags(status, bad, kFull, (threadIdx.x & 31) == 0);
}

// Forward apply: filt [T][K], loglik [T] (may be null), chain smoothing
// aggregates; `pre` holds the inclusive tile prefixes from the spine.
template <int K, int NW, int CH>
__global__ void __launch_bounds__(NW * 32) filter_apply_kernel(const Const<K>* __restrict__ cg,
                                                               const float* __restrict__ lik, int64_t T,
                                                               float* __restrict__ filt, float* __restrict__ loglik,
                                                               Bufs b, const float* __restrict__ pre,
                                                               uint32_t* status) {
    __shared__ Smem<K, NW> sm;
    constexpr int NG = Smem<K, NW>::NG;
    load_pi(cg, sm.Pi, sm.PiT, sm.q1);
    __syncthreads();
    const int w = threadIdx.x / K, lane = glane<K>();
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t c = (int64_t)blockIdx.x * NG + w;
    Flags bad = 0u;
    if (c < nch) {
        const int64_t k0 = c * CH, k1 = (k0 + CH < T) ? k0 + CH : T;
        // incoming prefix: tile prefix (x) the chain's exclusive in-tile prefix
        const bool has_tile = blockIdx.x > 0, has_in = w > 0;
        float p = 0.f, L = 0.f;
        bool has = has_tile || has_in;
        if (has) {
            FRow<K> r;
            if (has_tile) {
                load_frow(pre + ((int64_t)blockIdx.x - 1) * Dims<K>::FREC, r);
                if (has_in) {
                    FRow<K> e;
                    load_frow(b.fexcl + c * Dims<K>::FREC, e);
                    put_frow(sm.slot[w], e);
                    __syncwarp(gmask<K>());
                    combine_row(r, sm.slot[w], bad);
                }
            } else {
                load_frow(b.fexcl + c * Dims<K>::FREC, r);
            }
            row0_state(r, p, L);
        }
        float comp = 0.f;
        float a[K];   // this lane's row of the chain's smoothing aggregate
        float* sacc = sm.slot[w];
        __syncwarp(gmask<K>());
#pragma unroll 1
        for (int64_t k = k0; k < k1; ++k) {
            float l[K];
            const float lm = lik_row(lik, k, l, bad);
            float lx = 0.f;
#pragma unroll
            for (int x = 0; x < K; ++x) lx = (lane == x) ? l[x] : lx;
            if (!has) {   // step 1
                float v = sm.q1[lane] * lx;
                const float s = group_sum<K>(v);
                bad |= !(s > 0.f);
                p = v / s;
                L = lm + __logf(s);
                has = true;
            } else {
                advance_step<K>(p, L, comp, sm.Pi, lx, lm, bad);
            }
            filt[k * K + lane] = p;
            if (loglik && lane == 0) loglik[k] = L;
            float e[K];
            if (k == T - 1) selem_last_row(e, p);
            else selem_row(e, p, sm.PiT, bad);
            if (k == k0) {
#pragma unroll
                for (int x = 0; x < K; ++x) a[x] = e[x];
            } else {       // a_k0 (x) ... (x) a_k = a_k ... a_k0: row z of e times the aggregate
                put_srow(sacc, a);
                __syncwarp(gmask<K>());
                matmul_row(e, sacc);
                __syncwarp(gmask<K>());
#pragma unroll
                for (int x = 0; x < K; ++x) a[x] = e[x];
            }
        }
        store_srow(b.schain + c * Dims<K>::SREC, a);
        bad |= !isfinite(p) || !isfinite(L);
    }
    report_flags(status, bad, kFull, (threadIdx.x & 31) == 0);
}

// Reverse reduce: scan position j = tile * NG + w covers chain nch - 1 - j.
template <int K, int NW>
__global__ void __launch_bounds__(NW * 32) smoother_reduce_kernel(int64_t nch, Bufs b, uint32_t* status) {
    constexpr int NG = NW * 32 / K;
    __shared__ __align__(16) float slot[NG][Dims<K>::SLOT];
    const int w = threadIdx.x / K;
    const int64_t j0 = (int64_t)blockIdx.x * NG;
    const int nvalid = (nch - j0 < NG) ? (int)(nch - j0) : NG;
    if (w < nvalid) {
        float a[K];
        load_srow(b.schain + (nch - 1 - (j0 + w)) * Dims<K>::SREC, a);
        put_srow(slot[w], a);
    }
    __syncthreads();
    if (w == 0) {
        float acc[K];
        smem_row<Dims<K>::Q>(slot[0], glane<K>(), acc);
#pragma unroll 1
        for (int t = 1; t < nvalid; ++t) {
            store_srow(b.sexcl + (j0 + t) * Dims<K>::SREC, acc);
            matmul_row(acc, slot[t]);   // scan order: (later in time) (x)_r (earlier) = acc . chain
        }
        store_srow(b.sspine0 + (int64_t)blockIdx.x * Dims<K>::SREC, acc);
    }
    (void)status;
}

// Reverse apply: smooth [T][K]; `pre` holds the inclusive tile suffixes.
template <int K, int NW, int CH>
__global__ void __launch_bounds__(NW * 32) smoother_apply_kernel(const Const<K>* __restrict__ cg,
                                                                 const float* __restrict__ filt, int64_t T,
                                                                 float* __restrict__ smooth, Bufs b,
                                                                 const float* __restrict__ pre, uint32_t* status) {
    __shared__ Smem<K, NW> sm;
    constexpr int NG = Smem<K, NW>::NG;
    load_pi(cg, sm.Pi, sm.PiT, sm.q1);
    __syncthreads();
    const int w = threadIdx.x / K, lane = glane<K>();
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t j = (int64_t)blockIdx.x * NG + w;   // scan position
    Flags bad = 0u;
    if (j < nch) {
        const int64_t c = nch - 1 - j;
        const int64_t k0 = c * CH, k1 = (k0 + CH < T) ? k0 + CH : T;
        const bool has_tile = blockIdx.x > 0, has_in = w > 0;
        float s = 0.f;
        bool has = has_tile || has_in;
        if (has) {
            float a[K];
            if (has_tile) {
                load_srow(pre + ((int64_t)blockIdx.x - 1) * Dims<K>::SREC, a);
                if (has_in) {
                    float e[K];
                    load_srow(b.sexcl + j * Dims<K>::SREC, e);
                    put_srow(sm.slot[w], e);
                    __syncwarp(gmask<K>());
                    matmul_row(a, sm.slot[w]);
                }
            } else {
                load_srow(b.sexcl + j * Dims<K>::SREC, a);
            }
            s = row0_vec(a);
        }
#pragma unroll 1
        for (int64_t k = k1 - 1; k >= k0; --k) {
            const float p = __ldg(filt + k * K + lane);
            if (!has) {   // k = T - 1: the smoothed marginal is the filtered one
                s = p;
                has = true;
            } else {
                sadvance_step<K>(s, p, sm.PiT, bad);
            }
            smooth[k * K + lane] = s;
        }
        bad |= !isfinite(s);
    }
    report_flags(status, bad, kFull, (threadIdx.x & 31) == 0);
}

template <int K>
__global__ void __launch_bounds__(64) prep_kernel(const float* __restrict__ pi, const float* __restrict__ Pi,
                                                  Const<K>* __restrict__ out, uint32_t* __restrict__ status) {
    const int t = threadIdx.x;
    Flags bad = 0u;
    for (int e = t; e < K * K; e += blockDim.x) {
        const float v = Pi[e];
        bad |= !(v >= 0.f) || !(v <= 3.0e38f);
        out->Pi[e] = v;
    }
    for (int x = t; x < K; x += blockDim.x) {
        float s = 0.f;
        for (int y = 0; y < K; ++y) s = fmaf(pi[y], Pi[y * K + x], s);
        bad |= !(s >= 0.f) || !(s <= 3.0e38f);
        out->q1[x] = s;
    }
    report_flags(status, bad, kFull, (t & 31) == 0);
}

}  // namespace hmmw
}  // namespace ks
