// ks_tscan.cuh -- forward and reverse scans for nx = 32 on the tensor-core
// operators of ks_tc.cuh, one warp per chain of CH consecutive steps.
//
// Each scan runs as three kinds of launch (the paper's block-level elements,
// Section III-C, one block per tile of NW chains):
//   reduce   each warp folds its chain into one block element; warp 0 then
//            combines the tile's chain totals in order, storing each warp's
//            exclusive in-tile prefix, and writes the tile aggregate;
//   spine    one Kogge-Stone level over the tile aggregates per launch
//            (log2 tiles launches, one warp per tile, no waiting on other
//            blocks); a left operand that is already a complete prefix is
//            applied in its prefix-state form;
//   apply    each warp starts from the prefix entering its chain and applies
//            its steps one by one, writing one posterior per step.
// The reverse scan stores each smoothing element (Lemma 5) in its reduce
// launch and reads it back in its apply launch, so Lemma 5's inverse is
// formed once per step.  Chain order in the reverse scan is last chain first;
// in time order the operator takes the earlier step on the left (Lemma 6).
#pragma once

#include "ks_scan.cuh"
#include "ks_tc.cuh"

namespace ks {
namespace tc {

// Global scratch of the scans: per chain its total and its exclusive in-tile
// prefix (a record each), two spine buffers of one record per tile, and the
// smoothing elements of every step (reverse scan only).
struct TBuf {
    float* chains;   // nchains x 2 records
    float* spine0;   // ntiles records
    float* spine1;   // ntiles records
    float* elems;    // T smoothing records
};

template <int N, int M, int NW, class Const>
struct TSmem {
    static constexpr int KW = 6;                 // buffers per warp
    Const c;
    float pool[NW * KW * TD<N>::MAT];
    float vs[NW * VS<N>::FLOATS];
    static_assert(NW * KW <= 32, "pool mask");
    static_assert(NW * KW >= 11, "the in-tile combine holds up to 11 buffers");
};

// Shared memory of a spine launch: KS buffers per warp.
template <int N, int NWS, int KS>
struct SpineSmem {
    float pool[NWS * KS * TD<N>::MAT];
    float vs[NWS * VS<N>::FLOATS];
};
constexpr int kSpineWarps = 2;
constexpr int kSpineBufF = 11;                   // i (3) + j (3) + 5 in the filter combine
constexpr int kSpineBufS = 6;                    // i (2) + j (2) + 2 in the smoother combine

template <int N>
KS_DEV void put_fe(Pool<N>& pool, const FE& e) {
    pool.put(e.A);
    pool.put(e.C);
    pool.put(e.J);
}
template <int N>
KS_DEV void put_se(Pool<N>& pool, const SE& e) {
    pool.put(e.E);
    pool.put(e.L);
}
KS_DEV void copy_record(float* dst, const float* src, int n) {
    for (int i = lane_id(); i < n; i += 32) dst[i] = __ldcg(src + i);
}

// ---------------------------------------------------------------- forward
template <int N, int M, int NW, int CH>
__global__ void __launch_bounds__(NW * 32) tfilter_reduce_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                                 const float* __restrict__ y, int64_t T, TBuf tb,
                                                                 uint32_t* status) {
    using SM = TSmem<N, M, NW, FConst<N, M>>;
    constexpr int MAT = TD<N>::MAT, KW = SM::KW, FR = Rec<N>::F;
    extern __shared__ __align__(16) char tsm[];
    SM& sm = *reinterpret_cast<SM*>(tsm);
    build_fconst<N, M>(*mcg, sm.c);
    __syncthreads();
    const FConst<N, M>& c = sm.c;
    const int tile = blockIdx.x;
    const int w = threadIdx.x >> 5;
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t ch = (int64_t)tile * NW + w;
    const int64_t left = nch - (int64_t)tile * NW;
    const int nvalid = left < NW ? (int)left : NW;
    const bool valid = w < nvalid;
    const int64_t k0 = ch * CH;
    VS<N> vs{sm.vs + w * VS<N>::FLOATS};
    Flags bad = 0u;

    // ---- chain fold
    if (valid) {
        Pool<N> pool{sm.pool + w * KW * MAT, (1u << KW) - 1u};
        FE acc{pool.get(bad), pool.get(bad), pool.get(bad)};
        if (k0 == 0) {
            first_elem<N, M>(*mcg, c, acc);
        } else {
            float wv[M];
            const float b = meas<N, M>(c, y + k0 * M, wv);
            expand_meas<N, M>(c, b, wv, acc);
        }
#pragma unroll 1
        for (int i = 1; i < CH; ++i) {
            const int64_t k = k0 + i;
            if (k >= T) break;
            float wv[M];
            const float b = meas<N, M>(c, y + k * M, wv);
            fcomb_meas<N, M, false>(acc, c, b, wv, pool, vs, bad);
        }
        gstore_fe<N>(tb.chains + (size_t)ch * 2 * FR, acc);
    }
    __syncthreads();

    // ---- in-tile combine (warp 0 with every warp's buffers)
    if (w == 0) {
        Pool<N> pool{sm.pool, (uint32_t)((1ull << (NW * KW)) - 1ull)};
        const float* T0 = tb.chains + (size_t)tile * NW * 2 * FR;
        FE run = gload_fe<N>(T0, pool, bad);
#pragma unroll 1
        for (int t = 1; t < nvalid; ++t) {
            float* cht = tb.chains + ((size_t)tile * NW + t) * 2 * FR;
            gstore_fe<N>(cht + FR, run);                     // E_t = T_0 (x) ... (x) T_{t-1}
            const FE j = gload_fe<N>(cht, pool, bad);
            const FE o = fcombine<N>(run, j, pool, vs, bad);
            put_fe(pool, run);
            put_fe(pool, j);
            run = o;
        }
        gstore_fe<N>(tb.spine0 + (size_t)tile * FR, run);
    }
    report_flags(status, bad, kFull, lane_id() == 0);
}

// dst[t] = src[t - s] (x) src[t] for t >= s, else src[t].  src[t - s] covers
// tiles from 0 when t - s < s: then it is a prefix state (A = 0) and the
// result is one too (only b and C are formed and stored).
template <int N, int NWS>
__global__ void __launch_bounds__(NWS * 32) tspine_filter_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                                 int ntiles, int s, uint32_t* status) {
    using SM = SpineSmem<N, NWS, kSpineBufF>;
    constexpr int FR = Rec<N>::F;
    extern __shared__ __align__(16) char tsm[];
    SM& sm = *reinterpret_cast<SM*>(tsm);
    const int w = threadIdx.x >> 5;
    const int t = blockIdx.x * NWS + w;
    if (t >= ntiles) return;                              // whole warps; no block barrier below
    float* o = dst + (size_t)t * FR;
    if (t < s) {
        copy_record(o, src + (size_t)t * FR, FR);
        return;
    }
    Pool<N> pool{sm.pool + w * kSpineBufF * TD<N>::MAT, (1u << kSpineBufF) - 1u};
    VS<N> vs{sm.vs + w * VS<N>::FLOATS};
    Flags bad = 0u;
    const float* a = src + (size_t)(t - s) * FR;
    const float* b = src + (size_t)t * FR;
    if (t - s < s) {
        FE st{nullptr, pool.get(bad), nullptr};
        gload_fstate<N>(st.C, a);
        const FE j = gload_fe<N>(b, pool, bad);
        fadvance<N>(st, j, pool, vs, bad);
        gstore_fstate<N>(o, st.C);
    } else {
        const FE i = gload_fe<N>(a, pool, bad);
        const FE j = gload_fe<N>(b, pool, bad);
        const FE r = fcombine<N>(i, j, pool, vs, bad);
        gstore_fe<N>(o, r);
    }
    report_flags(status, bad, kFull, lane_id() == 0);
}

// `pre`: the spine's inclusive prefixes (record t covers tiles 0..t).
template <int N, int M, int NW, int CH>
__global__ void __launch_bounds__(NW * 32) tfilter_apply_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                                const float* __restrict__ y, int64_t T,
                                                                float* __restrict__ fmean, float* __restrict__ fcov,
                                                                TBuf tb, const float* __restrict__ pre,
                                                                uint32_t* status) {
    using SM = TSmem<N, M, NW, FConst<N, M>>;
    constexpr int MAT = TD<N>::MAT, KW = SM::KW, FR = Rec<N>::F;
    extern __shared__ __align__(16) char tsm[];
    SM& sm = *reinterpret_cast<SM*>(tsm);
    build_fconst<N, M>(*mcg, sm.c);
    __syncthreads();
    const FConst<N, M>& c = sm.c;
    const int tile = blockIdx.x;
    const int w = threadIdx.x >> 5, r = lane_id();
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t ch = (int64_t)tile * NW + w;
    if (ch >= nch) return;                                // whole warps; no block barrier below
    const int64_t k0 = ch * CH;
    const float* chE = tb.chains + (size_t)ch * 2 * FR + FR;
    VS<N> vs{sm.vs + w * VS<N>::FLOATS};
    Flags bad = 0u;
    Pool<N> pool{sm.pool + w * KW * MAT, (1u << KW) - 1u};
    FE st{nullptr, pool.get(bad), nullptr};
    bool has = false;
    if (tile != 0) {
        gload_fstate<N>(st.C, pre + (size_t)(tile - 1) * FR);
        if (w >= 1) {
            const FE j = gload_fe<N>(chE, pool, bad);
            fadvance<N>(st, j, pool, vs, bad);
            put_fe(pool, j);
        }
        has = true;
    } else if (w >= 1) {
        gload_fstate<N>(st.C, chE);                       // starts with the first element: A = 0
        has = true;
    }
    float probe = 0.f;
#pragma unroll 1
    for (int i = 0; i < CH; ++i) {
        const int64_t k = k0 + i;
        if (k >= T) break;
        if (!has) {
            first_elem<N, M>(*mcg, c, st);
            has = true;
        } else {
            float wv[M];
            const float b = meas<N, M>(c, y + k * M, wv);
            fcomb_meas<N, M, true>(st, c, b, wv, pool, vs, bad);
        }
        gstore_mat<N>(fcov + (size_t)k * N * N, st.C);
        gstore_vec<N>(fmean + (size_t)k * N, vrow<N>(st.C));
        probe += vrow<N>(st.C)[r] + st.C[r * TD<N>::P + r];
    }
    bad |= !isfinite(probe);
    report_flags(status, bad, kFull, r == 0);
}

// ---------------------------------------------------------------- reverse
template <int N, int M, int NW, int CH>
__global__ void __launch_bounds__(NW * 32) tsmoother_reduce_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                                   const float* __restrict__ fmean,
                                                                   const float* __restrict__ fcov, int64_t T, TBuf tb,
                                                                   uint32_t* status) {
    using SM = TSmem<N, M, NW, SConst<N, M>>;
    constexpr int MAT = TD<N>::MAT, KW = SM::KW, SR = Rec<N>::S;
    extern __shared__ __align__(16) char tsm[];
    SM& sm = *reinterpret_cast<SM*>(tsm);
    build_sconst<N, M>(*mcg, sm.c);
    __syncthreads();
    const SConst<N, M>& c = sm.c;
    const int tile = blockIdx.x;
    const int w = threadIdx.x >> 5;
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t u = (int64_t)tile * NW + w;               // scan-order chain index
    const int64_t left = nch - (int64_t)tile * NW;
    const int nvalid = left < NW ? (int)left : NW;
    const bool valid = w < nvalid;
    const int64_t cblk = nch - 1 - u;                        // chain in time order
    const int64_t klo = cblk * CH;
    const int64_t khi = valid ? ((klo + CH < T ? klo + CH : T) - 1) : -1;
    VS<N> vs{sm.vs + w * VS<N>::FLOATS};
    Flags bad = 0u;

    // ---- chain fold: a_klo (x) ... (x) a_khi, from the latest step back
    if (valid) {
        Pool<N> pool{sm.pool + w * KW * MAT, (1u << KW) - 1u};
        SE run{nullptr, nullptr};
#pragma unroll 1
        for (int64_t k = khi; k >= klo; --k) {
            float* Pm = pool.get(bad);
            gload_mat<N>(Pm, fcov + (size_t)k * N * N);
            gload_vec<N>(vrow<N>(Pm), fmean + (size_t)k * N);
            cp_wait();
            const SE e = selem<N, M>(Pm, c, k == T - 1, pool, vs, bad);
            gstore_se<N>(tb.elems + (size_t)k * SR, e);
            if (k == khi) {
                run = e;
            } else {
                const SE o = scombine<N, false>(e, run, pool, bad);
                pool.put(e.E);
                put_se(pool, run);
                run = o;
            }
        }
        gstore_se<N>(tb.chains + (size_t)u * 2 * SR, run);
    }
    __syncthreads();

    // ---- in-tile combine (warp 0): E_t = T_{t-1} (x) ... (x) T_0 in time order
    if (w == 0) {
        Pool<N> pool{sm.pool, (uint32_t)((1ull << (NW * KW)) - 1ull)};
        const float* T0 = tb.chains + (size_t)tile * NW * 2 * SR;
        SE run = gload_se<N>(T0, pool, bad);
#pragma unroll 1
        for (int t = 1; t < nvalid; ++t) {
            float* cht = tb.chains + ((size_t)tile * NW + t) * 2 * SR;
            gstore_se<N>(cht + SR, run);
            const SE j = gload_se<N>(cht, pool, bad);
            const SE o = scombine<N, false>(j, run, pool, bad);
            pool.put(j.E);
            put_se(pool, run);
            run = o;
        }
        gstore_se<N>(tb.spine0 + (size_t)tile * SR, run);
    }
    report_flags(status, bad, kFull, lane_id() == 0);
}

// Scan order (tile 0 = latest time): dst[u] = src[u] (x) src[u - s] in time
// order for u >= s, else src[u].  src[u - s] reaches the sequence's end when
// u - s < s: then it is a suffix state (E = 0) and so is the result.
template <int N, int NWS>
__global__ void __launch_bounds__(NWS * 32) tspine_smoother_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                                   int ntiles, int s, uint32_t* status) {
    using SM = SpineSmem<N, NWS, kSpineBufS>;
    constexpr int SR = Rec<N>::S;
    extern __shared__ __align__(16) char tsm[];
    SM& sm = *reinterpret_cast<SM*>(tsm);
    const int w = threadIdx.x >> 5;
    const int u = blockIdx.x * NWS + w;
    if (u >= ntiles) return;                              // whole warps; no block barrier below
    float* o = dst + (size_t)u * SR;
    if (u < s) {
        copy_record(o, src + (size_t)u * SR, SR);
        return;
    }
    Pool<N> pool{sm.pool + w * kSpineBufS * TD<N>::MAT, (1u << kSpineBufS) - 1u};
    Flags bad = 0u;
    const float* later = src + (size_t)(u - s) * SR;
    const SE i = gload_se<N>(src + (size_t)u * SR, pool, bad);
    if (u - s < s) {
        float* st = pool.get(bad);
        gload_sstate<N>(st, later);
        const SE r = scombine<N, true>(i, SE{nullptr, st}, pool, bad);
        gstore_sstate<N>(o, r.L);
    } else {
        const SE j = gload_se<N>(later, pool, bad);
        const SE r = scombine<N, false>(i, j, pool, bad);
        gstore_se<N>(o, r);
    }
    report_flags(status, bad, kFull, lane_id() == 0);
}

// `pre`: the spine's inclusive suffixes (record u covers scan tiles 0..u).
template <int N, int M, int NW, int CH>
__global__ void __launch_bounds__(NW * 32) tsmoother_apply_kernel(int64_t T, float* __restrict__ smean,
                                                                  float* __restrict__ scov, TBuf tb,
                                                                  const float* __restrict__ pre, uint32_t* status) {
    using SM = TSmem<N, M, NW, SConst<N, M>>;
    constexpr int MAT = TD<N>::MAT, KW = SM::KW, SR = Rec<N>::S;
    extern __shared__ __align__(16) char tsm[];
    SM& sm = *reinterpret_cast<SM*>(tsm);
    const int tile = blockIdx.x;
    const int w = threadIdx.x >> 5, r = lane_id();
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t u = (int64_t)tile * NW + w;
    if (u >= nch) return;                                 // whole warps; no block barrier below
    const int64_t cblk = nch - 1 - u;
    const int64_t klo = cblk * CH;
    const int64_t khi = (klo + CH < T ? klo + CH : T) - 1;
    const float* chE = tb.chains + (size_t)u * 2 * SR + SR;
    Flags bad = 0u;
    Pool<N> pool{sm.pool + w * KW * MAT, (1u << KW) - 1u};
    float* st = nullptr;                                  // L (g) of the running suffix
    if (tile != 0) {
        st = pool.get(bad);
        gload_sstate<N>(st, pre + (size_t)(tile - 1) * SR);
        if (w >= 1) {
            const SE j = gload_se<N>(chE, pool, bad);
            const SE o = scombine<N, true>(j, SE{nullptr, st}, pool, bad);
            pool.put(j.E);
            pool.put(st);
            st = o.L;
        }
    } else if (w >= 1) {
        st = pool.get(bad);
        gload_sstate<N>(st, chE);                        // ends with the last element: E = 0
    }
    float probe = 0.f;
#pragma unroll 1
    for (int64_t k = khi; k >= klo; --k) {
        const SE e = gload_se<N>(tb.elems + (size_t)k * SR, pool, bad);
        if (st == nullptr) {
            pool.put(e.E);
            st = e.L;
        } else {
            const SE o = scombine<N, true>(e, SE{nullptr, st}, pool, bad);
            pool.put(e.E);
            pool.put(st);
            st = o.L;
        }
        gstore_mat<N>(scov + (size_t)k * N * N, st);
        gstore_vec<N>(smean + (size_t)k * N, vrow<N>(st));
        probe += vrow<N>(st)[r] + st[r * TD<N>::P + r];
    }
    bad |= !isfinite(probe);
    report_flags(status, bad, kFull, r == 0);
}

}  // namespace tc
}  // namespace ks
