// ks_shard.cuh -- one aggregate element per time shard, for scans split along
// time across devices (the paper's block-level elements, Section III-C, with
// one block per device).
//
// A shard's filtering aggregate is a_s (x) ... (x) a_e over its steps
// (Lemma 4, earlier element on the left); its smoothing aggregate is the same
// fold of its Lemma 5 elements (Lemma 6).  Each thread folds CH consecutive
// steps, each thread block reduces its threads' folds in thread order, and a
// one-block pass reduces the blocks' results in block order, so the result is
// the ordered fold of all steps.  Elements are written in the packed layout
// of the operator batches (include/ks.h), so aggregates exchanged between
// devices combine with ks_filter_combine_batch / ks_smoother_combine_batch.
#pragma once

#include "ks_scan.cuh"

namespace ks {

template <int N>
KS_DEV void store_packed_f(float* o, const FElem<N>& r) {
#pragma unroll
    for (int a = 0; a < N * N; ++a) o[a] = r.A[a];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        o[N * N + a] = r.b[a];
        o[2 * N * N + N + a] = r.eta[a];
    }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            o[N * N + N + a * N + b] = r.C[sidx(a, b)];
            o[2 * N * N + 2 * N + a * N + b] = r.J[sidx(a, b)];
        }
}

template <int N>
KS_DEV SElem<N> load_packed_s(const float* p) {
    SElem<N> e;
#pragma unroll
    for (int a = 0; a < N * N; ++a) e.E[a] = p[a];
#pragma unroll
    for (int a = 0; a < N; ++a) e.g[a] = p[N * N + a];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) e.L[sidx(a, b)] = 0.5f * (p[N * N + N + a * N + b] + p[N * N + N + b * N + a]);
    return e;
}

template <int N>
KS_DEV void store_packed_s(float* o, const SElem<N>& c) {
#pragma unroll
    for (int a = 0; a < N * N; ++a) o[a] = c.E[a];
#pragma unroll
    for (int a = 0; a < N; ++a) o[N * N + a] = c.g[a];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) o[N * N + N + a * N + b] = c.L[sidx(a, b)];
}

// Lemma 4 / Lemma 6 in time order (earlier element on the left), with the
// packed-layout load/store of each.
template <int N>
struct FilterFold {
    using Elem = FElem<N>;
    static constexpr int SZ = 3 * N * N + 2 * N;
    KS_DEV static Elem combine(const Elem& a, const Elem& b, Flags& bad) { return fcombine<N>(a, b, bad); }
    KS_DEV static void identity(Elem& e) { set_identity<N>(e); }
    KS_DEV static Elem load(const float* p) { return load_packed_f<N>(p); }
    KS_DEV static void store(float* p, const Elem& e) { store_packed_f<N>(p, e); }
};
template <int N>
struct SmootherFold {
    using Elem = SElem<N>;
    static constexpr int SZ = 2 * N * N + N;
    KS_DEV static Elem combine(const Elem& a, const Elem& b, Flags&) { return scombine<N>(a, b); }
    KS_DEV static void identity(Elem& e) { set_identity<N>(e); }
    KS_DEV static Elem load(const float* p) { return load_packed_s<N>(p); }
    KS_DEV static void store(float* p, const Elem& e) { store_packed_s<N>(p, e); }
};

// The block's NT values combined in thread order; the result is in thread 0.
// Lane pairs at distance d = 1, 2, 4, ... combine (the left lane keeps the
// result), then thread 0 folds the warps' results in warp order.
template <class Op, int NT>
KS_DEV typename Op::Elem block_fold(typename Op::Elem x, typename Op::Elem* wsm, Flags& bad) {
    using E = typename Op::Elem;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const E o = shfl_down_t(x, d);
        if ((lane & (2 * d - 1)) == 0) x = Op::combine(x, o, bad);
    }
    if (lane == 0) wsm[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        x = wsm[0];
#pragma unroll 1
        for (int i = 1; i < NT / 32; ++i) x = Op::combine(x, wsm[i], bad);
    }
    return x;
}

// Filtering elements of steps [0, T) (Lemma 3 from y; the first one is the
// k = 1 element from (m0, P0) when `first`), folded per block into blk.
template <int N, int M, int NT, int CH>
__global__ void __launch_bounds__(NT) filter_fold_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                         const float* __restrict__ y, int64_t T, int first,
                                                         float* __restrict__ blk, uint32_t* status) {
    using Op = FilterFold<N>;
    __shared__ ModelConst<N, M> mc;
    __shared__ FElem<N> wsm[NT / 32];
    const int tid = threadIdx.x;
    load_const<N, M>(mcg, mc, tid, NT);
    __syncthreads();
    const int64_t k0 = ((int64_t)blockIdx.x * NT + tid) * CH;
    Flags bad = 0u;
    FElem<N> acc;
    if (k0 >= T) {
        set_identity<N>(acc);
    } else {
        if (k0 == 0 && first) {
            first_element<N, M>(mc, acc);
        } else {
            float yk[M], b[N], w[M];
            load_meas<M>(y, k0, yk);
            meas_element<N, M>(mc, yk, b, w);
            expand_meas<N, M>(mc, b, w, acc);
        }
#pragma unroll 1
        for (int i = 1; i < CH; ++i) {
            const int64_t k = k0 + i;
            if (k >= T) break;
            float yk[M], b[N], w[M];
            load_meas<M>(y, k, yk);
            meas_element<N, M>(mc, yk, b, w);
            acc = fcombine_meas<N, M>(acc, mc, b, w, bad);
        }
    }
    acc = block_fold<Op, NT>(acc, wsm, bad);
    if (tid == 0) Op::store(blk + (int64_t)blockIdx.x * Op::SZ, acc);
    report_flags(status, bad, kFull, (tid & 31) == 0);
}

// Smoothing elements of steps [0, T) from the filtered moments (Lemma 5; the
// last one is the k = n element when `last`), folded per block into blk.
template <int N, int M, int NT, int CH>
__global__ void __launch_bounds__(NT) smoother_fold_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                           const float* __restrict__ fmean,
                                                           const float* __restrict__ fcov, int64_t T, int last,
                                                           float* __restrict__ blk, uint32_t* status) {
    using Op = SmootherFold<N>;
    __shared__ ModelConst<N, M> mc;
    __shared__ SElem<N> wsm[NT / 32];
    const int tid = threadIdx.x;
    load_const<N, M>(mcg, mc, tid, NT);
    __syncthreads();
    const int64_t k0 = ((int64_t)blockIdx.x * NT + tid) * CH;
    Flags bad = 0u;
    SElem<N> acc;
    set_identity<N>(acc);
#pragma unroll 1
    for (int i = 0; i < CH; ++i) {
        const int64_t k = k0 + i;
        if (k >= T) break;
        float xb[N], P[sym_size(N)];
#pragma unroll
        for (int a = 0; a < N; ++a) xb[a] = __ldg(fmean + k * N + a);
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b)
                P[sidx(a, b)] = 0.5f * (__ldg(fcov + (k * N + a) * N + b) + __ldg(fcov + (k * N + b) * N + a));
        SElem<N> e;
        build_selem_from<N, M>(mc, xb, P, last && k == T - 1, e, bad);
        acc = (i == 0) ? e : scombine<N>(acc, e);
    }
    acc = block_fold<Op, NT>(acc, wsm, bad);
    if (tid == 0) Op::store(blk + (int64_t)blockIdx.x * Op::SZ, acc);
    report_flags(status, bad, kFull, (tid & 31) == 0);
}

// The nblk packed elements of blk folded in order into `out` (one block).
template <class Op, int NT>
__global__ void __launch_bounds__(NT) fold_packed_kernel(const float* __restrict__ blk, int nblk,
                                                         float* __restrict__ out, uint32_t* status) {
    __shared__ typename Op::Elem wsm[NT / 32];
    const int tid = threadIdx.x;
    const int per = (nblk + NT - 1) / NT;
    const int lo = tid * per, hi = lo + per < nblk ? lo + per : nblk;
    Flags bad = 0u;
    typename Op::Elem acc;
    Op::identity(acc);
#pragma unroll 1
    for (int i = lo; i < hi; ++i) {
        const typename Op::Elem e = Op::load(blk + (int64_t)i * Op::SZ);
        acc = (i == lo) ? e : Op::combine(acc, e, bad);
    }
    acc = block_fold<Op, NT>(acc, wsm, bad);
    if (tid == 0) Op::store(out, acc);
    report_flags(status, bad, kFull, (tid & 31) == 0);
}

}  // namespace ks
