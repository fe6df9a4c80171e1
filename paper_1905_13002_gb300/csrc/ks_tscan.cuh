// ks_tscan.cuh -- forward and reverse scans for nx = 32 on the tensor-core
// operators of ks_tc.cuh, one warp per chain of CH consecutive steps.
//
//   phase 1  each warp folds its chain into one block element (the block-level
//            elements of the paper's block decomposition);
//   phase 2  warp 0 alone, with every warp's buffers, combines the tile's
//            chain totals in order (storing each warp's exclusive in-tile
//            prefix), publishes the tile total and walks back over earlier
//            tiles (bounded waits) for the prefix entering the tile;
//   phase 3  each warp applies its steps one by one from its incoming prefix
//            and writes one posterior per step.
// The reverse scan stores each smoothing element (Lemma 5) in phase 1 and
// reads it back in phase 3, so Lemma 5's inverse is formed once per step.
// Chain order in the reverse scan is last chain first; in time order the
// operator takes the earlier step on the left (Lemma 6).
#pragma once

#include "ks_scan.cuh"
#include "ks_tc.cuh"

namespace ks {
namespace tc {

// Global scratch of the scans: per chain its total and its exclusive in-tile
// prefix (a record each), per tile the prefix entering it, and the smoothing
// elements of every step.
struct TBuf {
    float* chains;   // nchains x 2 records
    float* tex;      // ntiles records
    float* elems;    // T smoothing records (reverse scan only)
};

template <int N, int M, int NW, class Const>
struct TSmem {
    static constexpr int KW = 6;                 // buffers per warp
    Const c;
    float pool[NW * KW * TD<N>::MAT];
    float vs[NW * VS<N>::FLOATS];
    static_assert(NW * KW <= 32, "pool mask");
    static_assert(NW * KW >= 15, "the tile look-back holds up to 15 buffers");
};

KS_DEV void tpublish(uint32_t* flag, uint32_t v) {
    __threadfence();
    __syncwarp();
    if (lane_id() == 0) st_release(flag, v);
    __syncwarp();
}
KS_DEV uint32_t twait(const uint32_t* flag, uint32_t limit) {
    uint32_t f = 0u;
    if (lane_id() == 0) f = wait_flag(flag, limit);
    return __shfl_sync(kFull, f, 0);
}
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

// ---------------------------------------------------------------- forward
template <int N, int M, int NW, int CH>
__global__ void __launch_bounds__(NW * 32) tfilter_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                          const float* __restrict__ y, int64_t T,
                                                          float* __restrict__ fmean, float* __restrict__ fcov,
                                                          ScanState ss, TBuf tb) {
    using SM = TSmem<N, M, NW, FConst<N, M>>;
    constexpr int MAT = TD<N>::MAT, KW = SM::KW, FR = Rec<N>::F;
    extern __shared__ __align__(16) char tsm[];
    SM& sm = *reinterpret_cast<SM*>(tsm);
    __shared__ int s_tile;
    build_fconst<N, M>(*mcg, sm.c);
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(ss.counter, 1u);
    __syncthreads();
    const FConst<N, M>& c = sm.c;
    const int tile = s_tile;
    const int w = threadIdx.x >> 5, r = lane_id();
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t ch = (int64_t)tile * NW + w;
    const int64_t left = nch - (int64_t)tile * NW;
    const int nvalid = left < NW ? (int)left : NW;
    const bool valid = w < nvalid;
    const int64_t k0 = ch * CH;
    VS<N> vs{sm.vs + w * VS<N>::FLOATS};
    float* chT = tb.chains + (size_t)(valid ? ch : 0) * 2 * FR;
    float* chE = chT + FR;
    bool bad = false, lost = false;

    // ---- phase 1
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
        gstore_fe<N>(chT, acc);
    }
    __syncthreads();

    // ---- phase 2 (warp 0 with every warp's buffers)
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
        float* agg = ss.agg + (size_t)tile * FR;
        float* pre = ss.pre + (size_t)tile * FR;
        float* tex = tb.tex + (size_t)tile * FR;
        gstore_fe<N>(agg, run);
        if (tile == 0) {
            gstore_fe<N>(pre, run);
            tpublish(ss.flags, kFlagPre);
        } else {
            tpublish(ss.flags + tile, kFlagAgg);
            FE acc{nullptr, nullptr, nullptr};
            bool have = false;
            float* st = pool.get(bad);                        // the prefix entering the tile
#pragma unroll 1
            for (int j = tile - 1;; --j) {
                const uint32_t f = twait(ss.flags + j, ss.spin_limit);
                if (f == 0u) {
                    lost = true;
                    zero_mat<N>(st);
                    vrow<N>(st)[r] = 0.f;
                    break;
                }
                if (f == kFlagPre) {                          // published by another block: L2 loads
                    gload_fstate<N>(st, ss.pre + (size_t)j * FR);
                    if (have) {
                        FE s{nullptr, st, nullptr};
                        fadvance<N>(s, acc, pool, vs, bad);
                        put_fe(pool, acc);
                    }
                    break;
                }
                const FE aj = gload_fe<N>(ss.agg + (size_t)j * FR, pool, bad);
                if (have) {                                   // acc = AGG_j (x) acc (AGG_j is earlier)
                    const FE o = fcombine<N>(aj, acc, pool, vs, bad);
                    put_fe(pool, aj);
                    put_fe(pool, acc);
                    acc = o;
                } else {
                    acc = aj;
                    have = true;
                }
            }
            __syncwarp();
            gstore_fstate<N>(tex, st);
            FE s{nullptr, st, nullptr};
            fadvance<N>(s, run, pool, vs, bad);               // prefix through this tile
            gstore_fstate<N>(pre, st);
            tpublish(ss.flags + tile, kFlagPre);
        }
    }
    __syncthreads();

    // ---- phase 3
    if (valid) {
        Pool<N> pool{sm.pool + w * KW * MAT, (1u << KW) - 1u};
        FE st{nullptr, pool.get(bad), nullptr};
        bool has = false;
        if (tile != 0) {
            gload_fstate<N>(st.C, tb.tex + (size_t)tile * FR);
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
    }
    if (lost && r == 0) atomicOr(ss.status, ST_TIMEOUT);
    if (__any_sync(kFull, bad) && r == 0) atomicOr(ss.status, ST_NUMERIC);
}

// ---------------------------------------------------------------- reverse
template <int N, int M, int NW, int CH>
__global__ void __launch_bounds__(NW * 32) tsmoother_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                            const float* __restrict__ fmean,
                                                            const float* __restrict__ fcov, int64_t T,
                                                            float* __restrict__ smean, float* __restrict__ scov,
                                                            ScanState ss, TBuf tb) {
    using SM = TSmem<N, M, NW, SConst<N, M>>;
    constexpr int MAT = TD<N>::MAT, KW = SM::KW, SR = Rec<N>::S;
    extern __shared__ __align__(16) char tsm[];
    SM& sm = *reinterpret_cast<SM*>(tsm);
    __shared__ int s_tile;
    build_sconst<N, M>(*mcg, sm.c);
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(ss.counter, 1u);
    __syncthreads();
    const SConst<N, M>& c = sm.c;
    const int tile = s_tile;
    const int w = threadIdx.x >> 5, r = lane_id();
    const int64_t nch = (T + CH - 1) / CH;
    const int64_t u = (int64_t)tile * NW + w;               // scan-order chain index
    const int64_t left = nch - (int64_t)tile * NW;
    const int nvalid = left < NW ? (int)left : NW;
    const bool valid = w < nvalid;
    const int64_t cblk = nch - 1 - u;                        // chain in time order
    const int64_t klo = cblk * CH;
    const int64_t khi = valid ? ((klo + CH < T ? klo + CH : T) - 1) : -1;
    VS<N> vs{sm.vs + w * VS<N>::FLOATS};
    float* chT = tb.chains + (size_t)(valid ? u : 0) * 2 * SR;
    float* chE = chT + SR;
    bool bad = false, lost = false;

    // ---- phase 1: a_klo (x) ... (x) a_khi, folded from the latest step back
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
        gstore_se<N>(chT, run);
    }
    __syncthreads();

    // ---- phase 2 (warp 0; scan order: chain u covers later time than chain u + 1)
    if (w == 0) {
        Pool<N> pool{sm.pool, (uint32_t)((1ull << (NW * KW)) - 1ull)};
        const float* T0 = tb.chains + (size_t)tile * NW * 2 * SR;
        SE run = gload_se<N>(T0, pool, bad);
#pragma unroll 1
        for (int t = 1; t < nvalid; ++t) {                   // E_t = T_{t-1} (x) ... (x) T_0 in time order
            float* cht = tb.chains + ((size_t)tile * NW + t) * 2 * SR;
            gstore_se<N>(cht + SR, run);
            const SE j = gload_se<N>(cht, pool, bad);
            const SE o = scombine<N, false>(j, run, pool, bad);
            pool.put(j.E);
            put_se(pool, run);
            run = o;
        }
        float* agg = ss.agg + (size_t)tile * SR;
        float* pre = ss.pre + (size_t)tile * SR;
        float* tex = tb.tex + (size_t)tile * SR;
        gstore_se<N>(agg, run);
        if (tile == 0) {
            gstore_se<N>(pre, run);
            tpublish(ss.flags, kFlagPre);
        } else {
            tpublish(ss.flags + tile, kFlagAgg);
            SE acc{nullptr, nullptr};
            bool have = false;
            float* st = nullptr;                             // L (g) of the suffix entering the tile
#pragma unroll 1
            for (int j = tile - 1;; --j) {
                const uint32_t f = twait(ss.flags + j, ss.spin_limit);
                if (f == 0u) {
                    lost = true;
                    if (have) put_se(pool, acc);
                    st = pool.get(bad);
                    zero_mat<N>(st);
                    vrow<N>(st)[r] = 0.f;
                    break;
                }
                if (f == kFlagPre) {                          // published by another block: L2 loads
                    float* pj = pool.get(bad);
                    gload_sstate<N>(pj, ss.pre + (size_t)j * SR);
                    if (have) {                               // acc (x) PRE_j (PRE_j is later)
                        const SE o = scombine<N, true>(acc, SE{nullptr, pj}, pool, bad);
                        pool.put(acc.E);
                        pool.put(pj);
                        st = o.L;
                    } else {
                        st = pj;
                    }
                    break;
                }
                const SE aj = gload_se<N>(ss.agg + (size_t)j * SR, pool, bad);
                if (have) {                                   // acc = acc (x) AGG_j (AGG_j is later)
                    const SE o = scombine<N, false>(acc, aj, pool, bad);
                    pool.put(acc.E);
                    put_se(pool, aj);
                    acc = o;
                } else {
                    acc = aj;
                    have = true;
                }
            }
            __syncwarp();
            gstore_sstate<N>(tex, st);
            const SE o = scombine<N, true>(run, SE{nullptr, st}, pool, bad);   // run's L now holds it
            gstore_sstate<N>(pre, o.L);
            tpublish(ss.flags + tile, kFlagPre);
        }
    }
    __syncthreads();

    // ---- phase 3
    if (valid) {
        Pool<N> pool{sm.pool + w * KW * MAT, (1u << KW) - 1u};
        float* st = nullptr;                                 // L (g) of the running suffix
        if (tile != 0) {
            st = pool.get(bad);
            gload_sstate<N>(st, tb.tex + (size_t)tile * SR);
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
    }
    if (lost && r == 0) atomicOr(ss.status, ST_TIMEOUT);
    if (__any_sync(kFull, bad) && r == 0) atomicOr(ss.status, ST_NUMERIC);
}

}  // namespace tc
}  // namespace ks
