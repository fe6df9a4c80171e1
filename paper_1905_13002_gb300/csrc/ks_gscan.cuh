// ks_gscan.cuh -- forward and reverse scans for larger state sizes, one warp
// per chain of CH consecutive steps (elements in shared-memory slots, see
// ks_group.cuh).  Same three phases as ks_scan.cuh:
//   phase 1  each warp folds its chain into one block element;
//   phase 2  warps of a tile combine the chain totals in order (through
//            global scratch, so a warp needs only two element slots), the
//            warp that owns the tile total publishes it and walks back over
//            earlier tiles (bounded waits) for the prefix entering the tile;
//   phase 3  each warp applies its elements one by one from its incoming
//            posterior and writes one posterior per step (lane r: row r).
#pragma once

#include "ks_group.cuh"
#include "ks_scan.cuh"

namespace ks {
namespace grp {

// Global scratch of one scan: per chain its total and its exclusive in-tile
// prefix, per tile the exclusive prefix entering it (slot layout each).
struct GBuf {
    float* chains;   // nchains x 2 x slot
    float* tex;      // ntiles x slot
};

// Each lane publishes its rows, then lane 0 releases the flag: every lane's
// writes are fenced before the warp barrier that precedes the release.
KS_DEV void publish_flag(uint32_t* flag, uint32_t v) {
    __threadfence();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) st_release(flag, v);
    __syncwarp();
}

KS_DEV uint32_t warp_wait_flag(const uint32_t* flag, uint32_t limit) {
    uint32_t f = 0u;
    if ((threadIdx.x & 31) == 0) f = wait_flag(flag, limit);
    return __shfl_sync(kFullMask, f, 0);
}

// Copy an element slot (n floats) between two locations, warp-cooperatively.
KS_DEV void copy_floats(float* dst, const float* src, int n) {
    for (int i = threadIdx.x & 31; i < n; i += 32) dst[i] = src[i];
    __syncwarp();
}
KS_DEV void copy_floats_cg(float* dst, const float* src, int n) {
    for (int i = threadIdx.x & 31; i < n; i += 32) dst[i] = __ldcg(src + i);
    __syncwarp();
}

template <int N, int M>
KS_DEV void load_const_all(const ModelConst<N, M>* __restrict__ g, ModelConst<N, M>& s) {
    const float* src = reinterpret_cast<const float*>(g);
    float* dst = reinterpret_cast<float*>(&s);
    for (int i = threadIdx.x; i < (int)(sizeof(ModelConst<N, M>) / 4); i += blockDim.x) dst[i] = __ldg(src + i);
}

template <int N, int M, int NW>
struct GSmem {
    static constexpr int FS = Dim<N>::FSLOT, SS = Dim<N>::SSLOT;
    static constexpr int SLOT = FS > SS ? FS : SS;
    static constexpr int WARP = 3 * SLOT + Scratch<N>::FLOATS;      // three element slots + scratch
    static constexpr int BYTES = (int)sizeof(ModelConst<N, M>) + NW * WARP * 4 + 16;
    static KS_DEV ModelConst<N, M>& mc(char* base) { return *reinterpret_cast<ModelConst<N, M>*>(base); }
    static KS_DEV float* warp(char* base, int w) {
        return reinterpret_cast<float*>(base + ((sizeof(ModelConst<N, M>) + 15) / 16) * 16) + w * WARP;
    }
};

// ---------------------------------------------------------------- forward
template <int N, int M, int NW, int CH, bool SEG>
__global__ void __launch_bounds__(NW * 32) gfilter_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                          const float* __restrict__ y, int64_t T,
                                                          float* __restrict__ fmean, float* __restrict__ fcov,
                                                          ScanState ss, GBuf gb, Segs<N, M> segs) {
    using SM = GSmem<N, M, NW>;
    constexpr int FS = Dim<N>::FSLOT;
    extern __shared__ __align__(16) char gsm[];
    __shared__ int s_tile;
    ModelConst<N, M>& mc = SM::mc(gsm);
    load_const_all<N, M>(mcg, mc);
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(ss.counter, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int w = threadIdx.x >> 5, r = threadIdx.x & 31;
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t c = (int64_t)tile * NW + w;
    const int64_t left = nch - (int64_t)tile * NW;
    const int nvalid = left < NW ? (int)left : NW;
    const bool valid = w < nvalid;
    const int64_t k0 = c * CH;
    float* wb = SM::warp(gsm, w);
    FSlot<N> X[3] = {FSlot<N>{wb}, FSlot<N>{wb + SM::SLOT}, FSlot<N>{wb + 2 * SM::SLOT}};
    Scratch<N> s{wb + 3 * SM::SLOT};
    float* chT = gb.chains + (size_t)c * 2 * FS;        // chain total
    float* chE = chT + FS;                               // exclusive in-tile prefix
    bool bad = false, lost = false;
    Cursor<N, M, SEG> cur;

    // ---- phase 1
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
        wsync();
#pragma unroll 1
        for (int i = 1; i < CH; ++i) {
            const int64_t k = k0 + i;
            if (k >= T) break;
            cur.forward(segs, k);
            if (cur.first(k)) {
                reset_first<N, M>(r, *cur.mc, X[a]);
                wsync();
            } else {
                float wv[M];
                const float b = meas<N, M>(r, *cur.mc, y + k * M, wv);
                fcombine_meas<N, M, false>(r, X[a], *cur.mc, b, wv, X[a ^ 1], s, bad);
                a ^= 1;
            }
        }
        copy_floats(chT, X[a].p, FS);
    }
    __threadfence_block();
    __syncthreads();

    // ---- phase 2: in-tile exclusive prefixes, tile total, look-back
    const int L = nvalid - 1;          // warp that forms the tile total
    if (valid && (w >= 1 || w == L)) {
        const float* T0 = gb.chains + (size_t)(tile * NW) * 2 * FS;
        int a = 0;
        copy_floats_cg(X[0].p, T0, FS);
#pragma unroll 1
        for (int t = 1; t < w; ++t) {                    // operands staged in shared memory
            copy_floats_cg(X[2].p, T0 + (size_t)t * 2 * FS, FS);
            fcombine<N>(r, X[a], X[2], X[a ^ 1], s, bad);
            a ^= 1;
        }
        if (w >= 1) copy_floats(chE, X[a].p, FS);        // E_w = T_0 (x) ... (x) T_{w-1}
        if (w == L) {
            float* agg = ss.agg + (size_t)tile * FS;
            if (w >= 1) {
                copy_floats_cg(X[2].p, chT, FS);
                fcombine<N>(r, X[a], X[2], X[a ^ 1], s, bad);
                a ^= 1;
            }
            copy_floats(agg, X[a].p, FS);
            float* tex = gb.tex + (size_t)tile * FS;
            float* pre = ss.pre + (size_t)tile * FS;
            if (tile == 0) {
                copy_floats(pre, agg, FS);
                publish_flag(ss.flags, kFlagPre);
            } else {
                publish_flag(ss.flags + tile, kFlagAgg);
                bool have_run = false;
                int b = 0;
                int j = tile - 1;
#pragma unroll 1
                while (true) {
                    const uint32_t f = warp_wait_flag(ss.flags + j, ss.spin_limit);
                    if (f == 0u) {
                        lost = true;
                        for (int i = r; i < FS; i += 32) tex[i] = 0.f;
                        __syncwarp();
                        break;
                    }
                    if (f == kFlagPre) {     // published by another block: staged with L2 loads
                        float* pj = ss.pre + (size_t)j * FS;
                        if (have_run) {
                            copy_floats_cg(X[2].p, pj, FS);
                            fadvance<N>(r, X[2], X[b], FSlot<N>{tex}, s, bad);
                        } else {
                            copy_floats_cg(tex, pj, FS);
                        }
                        break;
                    }
                    float* aj = ss.agg + (size_t)j * FS;
                    if (have_run) {
                        copy_floats_cg(X[2].p, aj, FS);
                        fcombine<N>(r, X[2], X[b], X[b ^ 1], s, bad);
                        b ^= 1;
                    } else {
                        copy_floats_cg(X[b].p, aj, FS);
                        have_run = true;
                    }
                    --j;
                }
                __threadfence_block();
                copy_floats(X[2].p, tex, FS);
                copy_floats(X[0].p, agg, FS);
                fadvance<N>(r, X[2], X[0], X[1], s, bad);
                copy_floats(pre, X[1].p, FS);
                publish_flag(ss.flags + tile, kFlagPre);
            }
        }
    }
    __threadfence_block();
    __syncthreads();

    // ---- phase 3
    if (valid) {
        int a = 0;
        bool has = false;
        if (tile != 0) {
            const float* tex = gb.tex + (size_t)tile * FS;
            if (w >= 1) {
                copy_floats(X[2].p, tex, FS);
                copy_floats(X[1].p, chE, FS);
                fadvance<N>(r, X[2], X[1], X[0], s, bad);
            } else {
                copy_floats(X[0].p, tex, FS);
            }
            has = true;
        } else if (w >= 1) {
            copy_floats(X[0].p, chE, FS);        // E_w has A = 0 (it starts with the first element)
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
    }
    if (lost && r == 0) atomicOr(ss.status, ST_TIMEOUT);
    if (__any_sync(kFullMask, bad) && r == 0) atomicOr(ss.status, ST_NUMERIC);
}

// ---------------------------------------------------------------- reverse
// Chains are the forward blocks of CH steps, visited last first; in scan
// order x (x)_r y = y (x) x (Lemma 6, earlier time step on the left).
template <int N, int M, int NW, int CH, bool SEG>
__global__ void __launch_bounds__(NW * 32) gsmoother_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                            const float* __restrict__ fmean,
                                                            const float* __restrict__ fcov, int64_t T,
                                                            float* __restrict__ smean, float* __restrict__ scov,
                                                            ScanState ss, GBuf gb, Segs<N, M> segs) {
    using SM = GSmem<N, M, NW>;
    constexpr int SS = Dim<N>::SSLOT;
    extern __shared__ __align__(16) char gsm[];
    __shared__ int s_tile;
    ModelConst<N, M>& mc = SM::mc(gsm);
    load_const_all<N, M>(mcg, mc);
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(ss.counter, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int w = threadIdx.x >> 5, r = threadIdx.x & 31;
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t u = (int64_t)tile * NW + w;            // scan-order chain index
    const int64_t left = nch - (int64_t)tile * NW;
    const int nvalid = left < NW ? (int)left : NW;
    const bool valid = w < nvalid;
    const int64_t cblk = nch - 1 - u;                     // forward block
    const int64_t klo = cblk * CH;
    const int64_t khi = valid ? ((klo + CH < T ? klo + CH : T) - 1) : -1;
    float* wb = SM::warp(gsm, w);
    SSlot<N> X[3] = {SSlot<N>{wb}, SSlot<N>{wb + SM::SLOT}, SSlot<N>{wb + 2 * SM::SLOT}};
    Scratch<N> s{wb + 3 * SM::SLOT};
    float* chT = gb.chains + (size_t)u * 2 * SS;
    float* chE = chT + SS;
    bool bad = false, lost = false;
    Cursor<N, M, SEG> cur;

    // load the filtered posterior of step k into scratch S3 (rows) / V5
    auto load_post = [&](int64_t k) {
        if (r < N) {
            const float* src = fcov + (k * N + r) * N;
            float* dst = s.S(3) + r * Dim<N>::NP;
#pragma unroll Unroll<N>::K
            for (int q = 0; q < N; ++q) dst[q] = __ldg(src + q);
            s.V(5)[r] = __ldg(fmean + k * N + r);
        }
        wsync();
    };

    // ---- phase 1: a_{klo} (x) ... (x) a_{khi}, folded from the latest step back
    if (valid) {
        cur.seek(segs, &mc, khi, T);
        int a = 0;
        load_post(khi);
        selem<N, M>(r, *cur.mc, s.S(3), s.V(5), cur.last(khi), X[0], s, bad);
#pragma unroll 1
        for (int64_t k = khi - 1; k >= klo; --k) {
            cur.backward(segs, k);
            load_post(k);
            selem<N, M>(r, *cur.mc, s.S(3), s.V(5), cur.last(k), X[2], s, bad);
            scombine<N, false>(r, X[2], X[a], X[a ^ 1], s);
            a ^= 1;
        }
        copy_floats(chT, X[a].p, SS);
    }
    __threadfence_block();
    __syncthreads();

    // ---- phase 2 (scan order: chain u covers later time than chain u+1)
    const int L = nvalid - 1;
    if (valid && (w >= 1 || w == L)) {
        const float* T0 = gb.chains + (size_t)(tile * NW) * 2 * SS;
        int a = 0;
        copy_floats_cg(X[0].p, T0, SS);
#pragma unroll 1
        for (int t = 1; t < w; ++t) {       // E_w = T_{w-1} (x) ... (x) T_0 in time order
            copy_floats_cg(X[2].p, T0 + (size_t)t * 2 * SS, SS);
            scombine<N, false>(r, X[2], X[a], X[a ^ 1], s);
            a ^= 1;
        }
        if (w >= 1) copy_floats(chE, X[a].p, SS);
        if (w == L) {
            float* agg = ss.agg + (size_t)tile * SS;
            if (w >= 1) {
                copy_floats_cg(X[2].p, chT, SS);
                scombine<N, false>(r, X[2], X[a], X[a ^ 1], s);
                a ^= 1;
            }
            copy_floats(agg, X[a].p, SS);
            float* tex = gb.tex + (size_t)tile * SS;
            float* pre = ss.pre + (size_t)tile * SS;
            if (tile == 0) {
                copy_floats(pre, agg, SS);
                publish_flag(ss.flags, kFlagPre);
            } else {
                publish_flag(ss.flags + tile, kFlagAgg);
                bool have_run = false;
                int b = 0;
                int j = tile - 1;
#pragma unroll 1
                while (true) {
                    const uint32_t f = warp_wait_flag(ss.flags + j, ss.spin_limit);
                    if (f == 0u) {
                        lost = true;
                        for (int i = r; i < SS; i += 32) tex[i] = 0.f;
                        __syncwarp();
                        break;
                    }
                    if (f == kFlagPre) {     // published by another block: staged with L2 loads
                        float* pj = ss.pre + (size_t)j * SS;
                        if (have_run) {
                            copy_floats_cg(X[2].p, pj, SS);
                            scombine<N, true>(r, X[b], X[2], SSlot<N>{tex}, s);
                        } else {
                            copy_floats_cg(tex, pj, SS);
                        }
                        break;
                    }
                    float* aj = ss.agg + (size_t)j * SS;
                    if (have_run) {              // run = run (x) AGG_j in time order (AGG_j is later)
                        copy_floats_cg(X[2].p, aj, SS);
                        scombine<N, false>(r, X[b], X[2], X[b ^ 1], s);
                        b ^= 1;
                    } else {
                        copy_floats_cg(X[b].p, aj, SS);
                        have_run = true;
                    }
                    --j;
                }
                __threadfence_block();
                copy_floats(X[2].p, tex, SS);
                copy_floats(X[0].p, agg, SS);
                scombine<N, true>(r, X[0], X[2], X[1], s);
                copy_floats(pre, X[1].p, SS);
                publish_flag(ss.flags + tile, kFlagPre);
            }
        }
    }
    __threadfence_block();
    __syncthreads();

    // ---- phase 3
    if (valid) {
        int a = 0;
        bool has = false;
        if (tile != 0) {
            const float* tex = gb.tex + (size_t)tile * SS;
            if (w >= 1) {
                copy_floats(X[2].p, tex, SS);
                copy_floats(X[1].p, chE, SS);
                scombine<N, true>(r, X[1], X[2], X[0], s);
            } else {
                copy_floats(X[0].p, tex, SS);
            }
            has = true;
        } else if (w >= 1) {
            copy_floats(X[0].p, chE, SS);        // E = 0: it ends with the sequence's last element
            has = true;
        }
        cur.seek(segs, &mc, khi, T);
        float probe = 0.f;
#pragma unroll 1
        for (int64_t k = khi; k >= klo; --k) {
            cur.backward(segs, k);
            load_post(k);
            selem<N, M>(r, *cur.mc, s.S(3), s.V(5), cur.last(k), X[2], s, bad);
            if (!has) {
                copy_floats(X[a].p, X[2].p, SS);
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
    }
    if (lost && r == 0) atomicOr(ss.status, ST_TIMEOUT);
    if (__any_sync(kFullMask, bad) && r == 0) atomicOr(ss.status, ST_NUMERIC);
}

}  // namespace grp
}  // namespace ks
