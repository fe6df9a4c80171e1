// ks_gscan.cuh -- forward and reverse scans for larger state sizes, one lane
// group per chain of CH consecutive steps (elements in shared-memory slots,
// see ks_group.cuh: 8 lanes per chain for nx <= 8, a warp otherwise).  Each
// scan runs as three kinds of launch (the paper's block-level elements,
// Section III-C, one block per tile of NG chains):
//   reduce   each group folds its chain into one block element; group 0 then
//            combines the tile's chain totals in order, storing each chain's
//            exclusive in-tile prefix, and writes the tile aggregate;
//   spine    one Kogge-Stone level over the tile aggregates per launch
//            (log2 tiles launches, one group per tile, no waiting on other
//            blocks); a left operand that is already a complete prefix is
//            applied in its prefix-state form;
//   apply    each group starts from the prefix entering its chain and applies
//            its elements one by one, writing one posterior per step.
// With a full nx x nx combine (a pivoted inverse) per step of a cross-tile
// walk, a decoupled look-back kept most of each block waiting; the spine
// takes one combine per level instead.  Segmented batches need nothing in
// the spine: a sequence's first filtering element has A = 0 and its last
// smoothing element E = 0, so combines across a sequence start or end drop
// the other sequence exactly (the builders in reduce/apply know the segments).
#pragma once

#include "ks_group.cuh"
#include "ks_scan.cuh"

namespace ks {
namespace grp {

// Global scratch of one scan: per chain its total and its exclusive in-tile
// prefix (slot layout each), two spine buffers of one slot per tile, and (the
// reverse scan) every step's smoothing element, built once in reduce.
struct GBuf {
    float* chains;   // nchains x 2 x slot
    float* spine0;   // ntiles x slot
    float* spine1;   // ntiles x slot
    float* elems;    // T smoothing slots (reverse scan only)
};

// Copy an element slot (n floats) between two locations, by the lanes of the
// calling chain's group.
template <int N>
KS_DEV void copy_floats(float* dst, const float* src, int n) {
    constexpr int GS = Grp<N>::GS;
    for (int i = threadIdx.x & (GS - 1); i < n; i += GS) dst[i] = src[i];
    gsync<N>();
}
// The same from data written by other blocks or launches (L2 loads).
template <int N>
KS_DEV void copy_floats_cg(float* dst, const float* src, int n) {
    constexpr int GS = Grp<N>::GS;
    for (int i = threadIdx.x & (GS - 1); i < n; i += GS) dst[i] = __ldcg(src + i);
    gsync<N>();
}

template <int N, int M>
KS_DEV void load_const_all(const ModelConst<N, M>* __restrict__ g, ModelConst<N, M>& s) {
    const float* src = reinterpret_cast<const float*>(g);
    float* dst = reinterpret_cast<float*>(&s);
    for (int i = threadIdx.x; i < (int)(sizeof(ModelConst<N, M>) / 4); i += blockDim.x) dst[i] = __ldg(src + i);
}

// Per-chain buffer: three element slots and the scratch.  With 8-lane groups
// the stride is padded to 8 (mod 32) words, so the four groups of a warp
// reading their own row r (word 9 r + j + 8 g) or one broadcast row hit
// distinct banks.
template <int N>
struct GChain {
    static constexpr int FS = Dim<N>::FSLOT, SS = Dim<N>::SSLOT;
    static constexpr int SLOT = FS > SS ? FS : SS;
    static constexpr int RAW = 3 * SLOT + Scratch<N>::FLOATS;
    static constexpr int STRIDE = Grp<N>::GS == 32 ? RAW : RAW + ((8 - RAW % 32) + 32) % 32;
};

// Shared memory of a scan launch: the model constants and NW warps' chains.
template <int N, int M, int NW>
struct GSmem {
    static constexpr int SLOT = GChain<N>::SLOT;
    static constexpr int NG = NW * 32 / Grp<N>::GS;                  // chains per block
    static constexpr int BYTES = (int)sizeof(ModelConst<N, M>) + NG * GChain<N>::STRIDE * 4 + 16;
    static KS_DEV ModelConst<N, M>& mc(char* base) { return *reinterpret_cast<ModelConst<N, M>*>(base); }
    static KS_DEV float* chain(char* base, int g) {
        return reinterpret_cast<float*>(base + ((sizeof(ModelConst<N, M>) + 15) / 16) * 16) + g * GChain<N>::STRIDE;
    }
};

// Shared memory of a spine launch (no model constants): NWS warps' chains.
template <int N, int NWS>
struct GSpineSmem {
    static constexpr int NG = NWS * 32 / Grp<N>::GS;
    static constexpr int BYTES = NG * GChain<N>::STRIDE * 4;
    static KS_DEV float* chain(char* base, int g) { return reinterpret_cast<float*>(base) + g * GChain<N>::STRIDE; }
};
// Warps per spine block: up to 4, within 200 KB of shared memory.
template <int N>
constexpr int gspine_warps() {
    constexpr int per = GChain<N>::STRIDE * 4 * (32 / Grp<N>::GS);
    return per * 4 <= 200 * 1024 ? 4 : (200 * 1024 / per > 0 ? 200 * 1024 / per : 1);
}

// ---------------------------------------------------------------- forward
template <int N, int M, int NW, int CH, bool SEG, bool TV = false>
__global__ void __launch_bounds__(NW * 32) gfilter_reduce_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                                 const float* __restrict__ y, int64_t T, GBuf gb,
                                                                 uint32_t* status, Segs<N, M> segs) {
    using SM = GSmem<N, M, NW>;
    constexpr int FS = Dim<N>::FSLOT, NG = SM::NG;
    extern __shared__ __align__(16) char gsm[];
    ModelConst<N, M>& mc = SM::mc(gsm);
    load_const_all<N, M>(mcg, mc);
    __syncthreads();
    const int tile = blockIdx.x;
    const int w = threadIdx.x / Grp<N>::GS, r = threadIdx.x & (Grp<N>::GS - 1);
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t c = (int64_t)tile * NG + w;
    const int64_t left = nch - (int64_t)tile * NG;
    const int nvalid = left < NG ? (int)left : NG;
    const bool valid = w < nvalid;
    const int64_t k0 = c * CH;
    float* wb = SM::chain(gsm, w);
    FSlot<N> X[3] = {FSlot<N>{wb}, FSlot<N>{wb + SM::SLOT}, FSlot<N>{wb + 2 * SM::SLOT}};
    Scratch<N> s{wb + 3 * SM::SLOT};
    Flags bad = 0u;
    Cursor<N, M, SEG, TV> cur;

    // ---- chain fold
    if (valid) {
        cur.seek(segs, &mc, k0, T);
        int a = 0;
        if (cur.first(k0)) {
            first_elem<N, M>(r, *cur.mc, X[0]);
        } else {
            float wv[M];
            const float b = meas<N, M>(r, *cur.mc, y + k0 * M, wv);
            expand_meas<N, M>(r, *cur.mc, b, wv, X[0]);
        }
        gsync<N>();
#pragma unroll 1
        for (int i = 1; i < CH; ++i) {
            const int64_t k = k0 + i;
            if (k >= T) break;
            cur.forward(segs, k);
            if (cur.first(k)) {
                reset_first<N, M>(r, *cur.mc, X[a]);
                gsync<N>();
            } else {
                float wv[M];
                const float b = meas<N, M>(r, *cur.mc, y + k * M, wv);
                fcombine_meas<N, M, false>(r, X[a], *cur.mc, b, wv, X[a ^ 1], s, bad);
                a ^= 1;
            }
        }
        copy_floats<N>(gb.chains + (size_t)c * 2 * FS, X[a].p, FS);
    }
    __threadfence_block();
    __syncthreads();

    // ---- in-tile combine (warp 0)
    if (w == 0) {
        const float* T0 = gb.chains + (size_t)tile * NG * 2 * FS;
        int a = 0;
        copy_floats<N>(X[0].p, T0, FS);
#pragma unroll 1
        for (int t = 1; t < nvalid; ++t) {
            float* cht = gb.chains + ((size_t)tile * NG + t) * 2 * FS;
            copy_floats<N>(cht + FS, X[a].p, FS);              // E_t = T_0 (x) ... (x) T_{t-1}
            copy_floats<N>(X[2].p, cht, FS);
            fcombine<N>(r, X[a], X[2], X[a ^ 1], s, bad);
            a ^= 1;
        }
        copy_floats<N>(gb.spine0 + (size_t)tile * FS, X[a].p, FS);
    }
    report_flags(status, bad, gmask<N>(), r == 0);
}

// dst[t] = src[t - s] (x) src[t] for t >= s, else src[t].  src[t - s] covers
// tiles from 0 when t - s < s: then it is a prefix state (A = 0) and only b
// and C of the result are formed.
template <int N, int NWS>
__global__ void __launch_bounds__(NWS * 32) gspine_filter_kernel(const float* __restrict__ src, float* __restrict__ dst,
                                                                 int ntiles, int s, uint32_t* status) {
    using SM = GSpineSmem<N, NWS>;
    constexpr int FS = Dim<N>::FSLOT;
    constexpr int SLOT = GChain<N>::SLOT;
    extern __shared__ __align__(16) char gsm[];
    const int w = threadIdx.x / Grp<N>::GS, r = threadIdx.x & (Grp<N>::GS - 1);
    const int t = blockIdx.x * SM::NG + w;
    if (t >= ntiles) return;                              // whole warps; no block barrier below
    float* o = dst + (size_t)t * FS;
    if (t < s) {
        copy_floats_cg<N>(o, src + (size_t)t * FS, FS);
        return;
    }
    float* wb = SM::chain(gsm, w);
    FSlot<N> X[3] = {FSlot<N>{wb}, FSlot<N>{wb + SLOT}, FSlot<N>{wb + 2 * SLOT}};
    Scratch<N> sc{wb + 3 * SLOT};
    Flags bad = 0u;
    copy_floats_cg<N>(X[0].p, src + (size_t)(t - s) * FS, FS);
    copy_floats_cg<N>(X[1].p, src + (size_t)t * FS, FS);
    if (t - s < s) fadvance<N>(r, X[0], X[1], X[2], sc, bad);
    else fcombine<N>(r, X[0], X[1], X[2], sc, bad);
    copy_floats<N>(o, X[2].p, FS);
    report_flags(status, bad, gmask<N>(), r == 0);
}

// `pre`: the spine's inclusive prefixes (slot t covers tiles 0..t).
template <int N, int M, int NW, int CH, bool SEG, bool TV = false>
__global__ void __launch_bounds__(NW * 32) gfilter_apply_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                                const float* __restrict__ y, int64_t T,
                                                                float* __restrict__ fmean, float* __restrict__ fcov,
                                                                GBuf gb, const float* __restrict__ pre,
                                                                uint32_t* status, Segs<N, M> segs) {
    using SM = GSmem<N, M, NW>;
    constexpr int FS = Dim<N>::FSLOT, NG = SM::NG;
    extern __shared__ __align__(16) char gsm[];
    ModelConst<N, M>& mc = SM::mc(gsm);
    load_const_all<N, M>(mcg, mc);
    __syncthreads();
    const int tile = blockIdx.x;
    const int w = threadIdx.x / Grp<N>::GS, r = threadIdx.x & (Grp<N>::GS - 1);
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t c = (int64_t)tile * NG + w;
    if (c >= nch) return;                                 // whole warps; no block barrier below
    const int64_t k0 = c * CH;
    const float* chE = gb.chains + (size_t)c * 2 * FS + FS;
    float* wb = SM::chain(gsm, w);
    FSlot<N> X[3] = {FSlot<N>{wb}, FSlot<N>{wb + SM::SLOT}, FSlot<N>{wb + 2 * SM::SLOT}};
    Scratch<N> s{wb + 3 * SM::SLOT};
    Flags bad = 0u;
    Cursor<N, M, SEG, TV> cur;
    int a = 0;
    bool has = false;
    if (tile != 0) {
        const float* tex = pre + (size_t)(tile - 1) * FS;
        if (w >= 1) {
            copy_floats_cg<N>(X[2].p, tex, FS);
            copy_floats_cg<N>(X[1].p, chE, FS);
            fadvance<N>(r, X[2], X[1], X[0], s, bad);
        } else {
            copy_floats_cg<N>(X[0].p, tex, FS);
        }
        has = true;
    } else if (w >= 1) {
        copy_floats_cg<N>(X[0].p, chE, FS);                 // E_w has A = 0 (it starts with the first element)
        has = true;
    }
    cur.seek(segs, &mc, k0, T);
    float probe = 0.f;
#pragma unroll 1
    for (int i = 0; i < CH; ++i) {
        const int64_t k = k0 + i;
        if (k >= T) break;
        cur.forward(segs, k);
        if (cur.first(k) || !has) {
            first_state<N, M>(r, *cur.mc, X[a]);
            has = true;
        } else {
            float wv[M];
            const float b = meas<N, M>(r, *cur.mc, y + k * M, wv);
            fcombine_meas<N, M, true>(r, X[a], *cur.mc, b, wv, X[a ^ 1], s, bad);
            a ^= 1;
        }
        if (r < N) {
            const float bm = X[a].b()[r];
            fmean[k * N + r] = bm;
            float* crow = fcov + (k * N + r) * N;
            const float* src = X[a].C() + r * Dim<N>::NP;
#pragma unroll Unroll<N>::K
            for (int q = 0; q < N; ++q) crow[q] = src[q];
            probe += bm + src[r];
        }
    }
    bad |= !isfinite(probe);
    report_flags(status, bad, gmask<N>(), r == 0);
}

// ---------------------------------------------------------------- reverse
// Chains are the forward blocks of CH steps, visited last first; in time
// order the operator takes the earlier step on the left (Lemma 6).
template <int N, int M, int NW, int CH, bool SEG, bool TV = false>
__global__ void __launch_bounds__(NW * 32) gsmoother_reduce_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                                   const float* __restrict__ fmean,
                                                                   const float* __restrict__ fcov, int64_t T, GBuf gb,
                                                                   uint32_t* status, Segs<N, M> segs) {
    using SM = GSmem<N, M, NW>;
    constexpr int SS = Dim<N>::SSLOT, NG = SM::NG;
    extern __shared__ __align__(16) char gsm[];
    ModelConst<N, M>& mc = SM::mc(gsm);
    load_const_all<N, M>(mcg, mc);
    __syncthreads();
    const int tile = blockIdx.x;
    const int w = threadIdx.x / Grp<N>::GS, r = threadIdx.x & (Grp<N>::GS - 1);
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t u = (int64_t)tile * NG + w;            // scan-order chain index
    const int64_t left = nch - (int64_t)tile * NG;
    const int nvalid = left < NG ? (int)left : NG;
    const bool valid = w < nvalid;
    const int64_t cblk = nch - 1 - u;                     // forward block
    const int64_t klo = cblk * CH;
    const int64_t khi = valid ? ((klo + CH < T ? klo + CH : T) - 1) : -1;
    float* wb = SM::chain(gsm, w);
    SSlot<N> X[3] = {SSlot<N>{wb}, SSlot<N>{wb + SM::SLOT}, SSlot<N>{wb + 2 * SM::SLOT}};
    Scratch<N> s{wb + 3 * SM::SLOT};
    Flags bad = 0u;
    Cursor<N, M, SEG, TV> cur;

    // ---- chain fold: a_{klo} (x) ... (x) a_{khi}, from the latest step back
    if (valid) {
        auto load_post = [&](int64_t k) {
            if (r < N) {
                const float* src = fcov + (k * N + r) * N;
                float* dst = s.S(3) + r * Dim<N>::NP;
#pragma unroll Unroll<N>::K
                for (int q = 0; q < N; ++q) dst[q] = __ldg(src + q);
                s.V(5)[r] = __ldg(fmean + k * N + r);
            }
            gsync<N>();
        };
        cur.seek(segs, &mc, khi, T);
        int a = 0;
        load_post(khi);
        selem<N, M>(r, *cur.trans(khi), s.S(3), s.V(5), cur.last(khi), X[0], s, bad);
        copy_floats<N>(gb.elems + (size_t)khi * SS, X[0].p, SS);
#pragma unroll 1
        for (int64_t k = khi - 1; k >= klo; --k) {
            cur.backward(segs, k);
            load_post(k);
            selem<N, M>(r, *cur.trans(k), s.S(3), s.V(5), cur.last(k), X[2], s, bad);
            copy_floats<N>(gb.elems + (size_t)k * SS, X[2].p, SS);
            scombine<N, false>(r, X[2], X[a], X[a ^ 1], s);
            a ^= 1;
        }
        copy_floats<N>(gb.chains + (size_t)u * 2 * SS, X[a].p, SS);
    }
    __threadfence_block();
    __syncthreads();

    // ---- in-tile combine (warp 0): E_t = T_{t-1} (x) ... (x) T_0 in time order
    if (w == 0) {
        const float* T0 = gb.chains + (size_t)tile * NG * 2 * SS;
        int a = 0;
        copy_floats<N>(X[0].p, T0, SS);
#pragma unroll 1
        for (int t = 1; t < nvalid; ++t) {
            float* cht = gb.chains + ((size_t)tile * NG + t) * 2 * SS;
            copy_floats<N>(cht + SS, X[a].p, SS);
            copy_floats<N>(X[2].p, cht, SS);
            scombine<N, false>(r, X[2], X[a], X[a ^ 1], s);
            a ^= 1;
        }
        copy_floats<N>(gb.spine0 + (size_t)tile * SS, X[a].p, SS);
    }
    report_flags(status, bad, gmask<N>(), r == 0);
}

// Scan order (tile 0 = latest time): dst[u] = src[u] (x) src[u - s] in time
// order for u >= s, else src[u].  src[u - s] reaches the sequence's end when
// u - s < s: then it is a suffix state (E = 0) and only g and L are formed.
template <int N, int NWS>
__global__ void __launch_bounds__(NWS * 32) gspine_smoother_kernel(const float* __restrict__ src,
                                                                   float* __restrict__ dst, int ntiles, int s,
                                                                   uint32_t* status) {
    using SM = GSpineSmem<N, NWS>;
    constexpr int SS = Dim<N>::SSLOT;
    constexpr int SLOT = GChain<N>::SLOT;
    extern __shared__ __align__(16) char gsm[];
    const int w = threadIdx.x / Grp<N>::GS, r = threadIdx.x & (Grp<N>::GS - 1);
    const int u = blockIdx.x * SM::NG + w;
    if (u >= ntiles) return;                              // whole warps; no block barrier below
    float* o = dst + (size_t)u * SS;
    if (u < s) {
        copy_floats_cg<N>(o, src + (size_t)u * SS, SS);
        return;
    }
    float* wb = SM::chain(gsm, w);
    SSlot<N> X[3] = {SSlot<N>{wb}, SSlot<N>{wb + SLOT}, SSlot<N>{wb + 2 * SLOT}};
    Scratch<N> sc{wb + 3 * SLOT};
    copy_floats_cg<N>(X[0].p, src + (size_t)u * SS, SS);
    copy_floats_cg<N>(X[1].p, src + (size_t)(u - s) * SS, SS);
    if (u - s < s) scombine<N, true>(r, X[0], X[1], X[2], sc);
    else scombine<N, false>(r, X[0], X[1], X[2], sc);
    copy_floats<N>(o, X[2].p, SS);
    (void)status;
}

// `pre`: the spine's inclusive suffixes (slot u covers scan tiles 0..u).
// The smoothing elements come from the reduce launch (gb.elems).
template <int N, int M, int NW, int CH>
__global__ void __launch_bounds__(NW * 32) gsmoother_apply_kernel(int64_t T, float* __restrict__ smean,
                                                                  float* __restrict__ scov, GBuf gb,
                                                                  const float* __restrict__ pre, uint32_t* status) {
    using SM = GSmem<N, M, NW>;
    constexpr int SS = Dim<N>::SSLOT, NG = SM::NG;
    extern __shared__ __align__(16) char gsm[];
    const int tile = blockIdx.x;
    const int w = threadIdx.x / Grp<N>::GS, r = threadIdx.x & (Grp<N>::GS - 1);
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t u = (int64_t)tile * NG + w;
    if (u >= nch) return;                                 // whole warps; no block barrier in this kernel
    const int64_t cblk = nch - 1 - u;
    const int64_t klo = cblk * CH;
    const int64_t khi = (klo + CH < T ? klo + CH : T) - 1;
    const float* chE = gb.chains + (size_t)u * 2 * SS + SS;
    float* wb = SM::chain(gsm, w);
    SSlot<N> X[3] = {SSlot<N>{wb}, SSlot<N>{wb + SM::SLOT}, SSlot<N>{wb + 2 * SM::SLOT}};
    Scratch<N> s{wb + 3 * SM::SLOT};
    Flags bad = 0u;
    int a = 0;
    bool has = false;
    if (tile != 0) {
        const float* tex = pre + (size_t)(tile - 1) * SS;
        if (w >= 1) {
            copy_floats_cg<N>(X[2].p, tex, SS);
            copy_floats_cg<N>(X[1].p, chE, SS);
            scombine<N, true>(r, X[1], X[2], X[0], s);
        } else {
            copy_floats_cg<N>(X[0].p, tex, SS);
        }
        has = true;
    } else if (w >= 1) {
        copy_floats_cg<N>(X[0].p, chE, SS);                 // E = 0: it ends with the sequence's last element
        has = true;
    }
    float probe = 0.f;
#pragma unroll 1
    for (int64_t k = khi; k >= klo; --k) {
        copy_floats_cg<N>(X[2].p, gb.elems + (size_t)k * SS, SS);
        if (!has) {
            copy_floats<N>(X[a].p, X[2].p, SS);
            has = true;
        } else {
            scombine<N, true>(r, X[2], X[a], X[a ^ 1], s);
            a ^= 1;
        }
        if (r < N) {
            const float g = X[a].g()[r];
            smean[k * N + r] = g;
            float* lrow = scov + (k * N + r) * N;
            const float* src = X[a].L() + r * Dim<N>::NP;
#pragma unroll Unroll<N>::K
            for (int q = 0; q < N; ++q) lrow[q] = src[q];
            probe += g + src[r];
        }
    }
    bad |= !isfinite(probe);
    report_flags(status, bad, gmask<N>(), r == 0);
}

}  // namespace grp
}  // namespace ks
