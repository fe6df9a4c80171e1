// ks_impl.cuh -- host side of one (nx, ny) instantiation: workspace layout,
// argument checks and kernel launches behind the C ABI of include/ks.h.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/ks.h"
#include "ks_scan.cuh"
#include "ks_shard.cuh"

namespace ks {

// Polls of a look-back flag before a wait is declared lost (sleeps grow to
// ~1 us, so this is roughly one second).
constexpr uint32_t kSpinLimit = 1000000u;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
    int64_t T = 0, ld = 0;
    int B = 1;
    int ntf = 0, nts = 0;
    size_t off_const = 0, off_coef = 0, off_flags = 0, flags_bytes = 0;
    size_t off_fagg = 0, off_fpre = 0, off_sagg = 0, off_spre = 0, off_sblk = 0;
    size_t off_elems = 0, off_fmean = 0, off_fcov = 0;
    size_t bytes_smooth = 0, bytes_elements = 0;
};

// Function table of one instantiation.
struct VTable {
    int nx, ny;
    Layout (*layout)(int64_t T, int B);
    int (*build_elements)(const ks_model*, const float*, int64_t, void*, size_t, cudaStream_t);
    int (*filter_scan)(const ks_model*, int64_t, void*, size_t, float*, float*, cudaStream_t);
    int (*smooth_scan)(const ks_model*, int64_t, const float*, const float*, void*, size_t, float*, float*,
                       cudaStream_t);
    int (*smooth)(const ks_model*, const float*, int64_t, void*, size_t, float*, float*, float*, float*,
                  cudaStream_t, void* const*);
    int (*smooth_batch)(const ks_model_batch*, const float*, int64_t, void*, size_t, float*, float*, float*,
                        float*, cudaStream_t);
    int (*fcomb_batch)(int64_t, const float*, const float*, float*, void*, cudaStream_t);
    int (*scomb_batch)(int64_t, const float*, const float*, float*, void*, cudaStream_t);
    size_t (*agg_bytes)(int64_t T);
    int (*faggregate)(const ks_model*, const float*, int64_t, int, void*, size_t, float*, cudaStream_t);
    int (*saggregate)(const ks_model*, int64_t, const float*, const float*, int, void*, size_t, float*,
                      cudaStream_t);
    size_t (*tv_bytes)(int64_t T);   // workspace of a time-varying smooth (null: not supported)
};

// The fused end-to-end entry points of one steps-per-thread choice.
struct ChunkVariant {
    Layout (*layout)(int64_t T, int B);
    // the last argument: fold full blocks with the linear block fold
    int (*smooth)(const ks_model*, const float*, int64_t, void*, size_t, float*, float*, float*, float*,
                  cudaStream_t, void* const*, bool);
    int (*smooth_batch)(const ks_model_batch*, const float*, int64_t, void*, size_t, float*, float*, float*,
                        float*, cudaStream_t, bool);
};

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline int launch_status() {
    return cudaGetLastError() == cudaSuccess ? KS_OK : KS_ECUDA;
}

// Launch with programmatic stream serialization: the kernel may be scheduled
// while the previous kernel of the stream drains (it calls pdl_wait() before
// reading that kernel's results), which hides the launch gap between the
// preparation and the scans.
template <class... KArgs, class... Args>
inline int launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...) == cudaSuccess ? KS_OK : KS_ECUDA;
}

// FCH_ = steps per thread of the block scans (one tile = 128 * FCH_ steps).
template <int N, int M, int FCH_ = 32>
struct Impl {
    static constexpr int FNT = 128, FCH = FCH_;   // forward scan: threads, steps per thread
    static constexpr int SNT = 128, SCH = FCH;  // reverse scan (same block grid)
    static constexpr int64_t FTILE = (int64_t)FNT * FCH, STILE = (int64_t)SNT * SCH;
    static constexpr int NCOMP = 3 * N * N + 2 * N;   // scalars of one filtering element

    static constexpr size_t prep_smem() { return sizeof(PrepSmem<N, M>) + sizeof(ModelConst<N, M>) + 16; }

    static Layout layout(int64_t T, int B = 1) {
        Layout L;
        L.T = T;
        L.B = B;
        L.ld = (int64_t)align_up((size_t)T, 64);
        L.ntf = (int)((T + FTILE - 1) / FTILE);
        L.nts = (int)((T + STILE - 1) / STILE);
        size_t off = 256;                                   // status word + reserved
        L.off_const = off;                                  // one ModelConst per segment
        off = align_up(off + sizeof(ModelConst<N, M>) * (size_t)B, 256);
        L.off_coef = off;                                   // one BlockCoef per segment
        off = align_up(off + sizeof(BlockCoef<N, M>) * (size_t)B, 256);
        L.off_flags = off;   // [fcounter, scounter, retry counter, pad][fflags][sflags][retry fflags]
        L.flags_bytes = 16 + 4 * (size_t)(2 * L.ntf + L.nts);
        off = align_up(off + L.flags_bytes, 256);
        L.off_fagg = off;
        off = align_up(off + sizeof(FElem<N>) * (size_t)L.ntf, 256);
        L.off_fpre = off;
        off = align_up(off + sizeof(FState<N>) * (size_t)L.ntf, 256);
        L.off_sagg = off;
        off = align_up(off + sizeof(SElem<N>) * (size_t)L.nts, 256);
        L.off_spre = off;
        off = align_up(off + sizeof(SState<N>) * (size_t)L.nts, 256);
        L.off_sblk = off;                                   // smoothing aggregate per forward block
        off = align_up(off + sizeof(SElem<N>) * (size_t)((T + FCH - 1) / FCH), 256);
        L.bytes_smooth = off;
        L.off_elems = off;
        off = align_up(off + 4 * (size_t)NCOMP * (size_t)L.ld, 256);
        L.off_fmean = off;
        off = align_up(off + 4 * (size_t)N * (size_t)T, 256);
        L.off_fcov = off;
        off = align_up(off + 4 * (size_t)N * N * (size_t)T, 256);
        L.bytes_elements = off;
        return L;
    }

    static ModelConst<N, M>* mconst(void* ws, const Layout& L) {
        return reinterpret_cast<ModelConst<N, M>*>(static_cast<char*>(ws) + L.off_const);
    }
    static BlockCoef<N, M>* coef(void* ws, const Layout& L) {
        return reinterpret_cast<BlockCoef<N, M>*>(static_cast<char*>(ws) + L.off_coef);
    }
    static uint32_t* status(void* ws) { return static_cast<uint32_t*>(ws); }

    static ScanState fstate(void* ws, const Layout& L) {
        char* b = static_cast<char*>(ws);
        ScanState s;
        s.counter = reinterpret_cast<uint32_t*>(b + L.off_flags);
        s.flags = reinterpret_cast<uint32_t*>(b + L.off_flags + 16);
        s.agg = reinterpret_cast<float*>(b + L.off_fagg);
        s.pre = reinterpret_cast<float*>(b + L.off_fpre);
        s.status = status(ws);
        s.spin_limit = kSpinLimit;
        return s;
    }
    // The forward scan's retry with refinement: its own counter and flags.
    static ScanState fstate_retry(void* ws, const Layout& L) {
        ScanState s = fstate(ws, L);
        char* b = static_cast<char*>(ws);
        s.counter = reinterpret_cast<uint32_t*>(b + L.off_flags + 8);
        s.flags = reinterpret_cast<uint32_t*>(b + L.off_flags + 16 + 4 * (size_t)(L.ntf + L.nts));
        return s;
    }
    static ScanState sstate(void* ws, const Layout& L) {
        char* b = static_cast<char*>(ws);
        ScanState s;
        s.counter = reinterpret_cast<uint32_t*>(b + L.off_flags + 4);
        s.flags = reinterpret_cast<uint32_t*>(b + L.off_flags + 16 + 4 * (size_t)L.ntf);
        s.agg = reinterpret_cast<float*>(b + L.off_sagg);
        s.pre = reinterpret_cast<float*>(b + L.off_spre);
        s.status = status(ws);
        s.spin_limit = kSpinLimit;
        return s;
    }

    static int check_model(const ks_model* m) {
        if (!m || !m->F || !m->Q || !m->H || !m->R || !m->m0 || !m->P0) return KS_EINVAL;
        if (m->time_varying != 0) return KS_EUNSUPPORTED;
        return KS_OK;
    }

    static int check_common(const ks_model* m, int64_t T, void* ws, size_t ws_bytes, size_t need) {
        int rc = check_model(m);
        if (rc) return rc;
        if (T < 1 || T > 0x7fffffffLL) return KS_EINVAL;
        if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < need) return KS_EINVAL;
        return KS_OK;
    }

    // Model constants (and the k = 1 element when y is given, with the block
    // fold's coefficients when `fold` is set and the layout has room for
    // them); also zeroes the scans' tile counters and flags, which every scan
    // launch needs.
    static int prep(const ks_model* m, const float* y, void* ws, const Layout& L, cudaStream_t st,
                    bool fold = false) {
        uint32_t* z = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + L.off_flags);
        BlockCoef<N, M>* cf = (fold && y && L.off_coef) ? coef(ws, L) : nullptr;
        auto k = cf ? prep_kernel<N, M, true> : prep_kernel<N, M, false>;
        k<<<1, kPrepThreads, prep_smem(), st>>>(m->F, m->u, m->Q, m->H, m->d, m->R, m->m0, m->P0, y, mconst(ws, L),
                                                status(ws), z, (int)(L.flags_bytes / 4), nullptr, L.T,
                                                status(ws) + HDR_FIRST_TILE, cf, FCH);
        return launch_status();
    }

    static Segs<N, M> no_segs() { return Segs<N, M>{nullptr, nullptr, 1}; }

    static int reset_flags(void* ws, const Layout& L, cudaStream_t st) {
        return cudaMemsetAsync(static_cast<char*>(ws) + L.off_flags, 0, L.flags_bytes, st) == cudaSuccess
                   ? KS_OK : KS_ECUDA;
    }

    // Dynamic shared memory above 48 KB needs an explicit opt-in per kernel.
    template <class K>
    static bool allow_smem(K kernel, int bytes) {
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
    }

    static float* sblk(void* ws, const Layout& L) {
        return reinterpret_cast<float*>(static_cast<char*>(ws) + L.off_sblk);
    }

    template <bool SEG>
    static int launch_filter_fused(void* ws, const Layout& L, const float* y, float* fm, float* fc,
                                   Segs<N, M> segs, cudaStream_t st) {
        constexpr int smem = filter_dyn_smem<N, FNT>();
        auto k = filter_scan_kernel<N, M, FNT, FCH, true, true, SEG, false, REF_DETECT, false>;
        auto kr = filter_scan_kernel<N, M, FNT, FCH, true, true, SEG, false, REF_FP64, true>;
        static const bool ok = allow_smem(k, smem) && allow_smem(kr, smem);
        if (!ok) return KS_ECUDA;
        const ModelConst<N, M>* mc = mconst(ws, L);
        const float* none = nullptr;
        float* sb = sblk(ws, L);
        int rc = launch_pdl(k, L.ntf, FNT, smem, st, mc, y, none, L.ld, L.T, fm, fc, fstate(ws, L), sb, segs,
                            TVArgs{});
        if (rc) return rc;
        return launch_pdl(kr, L.ntf, FNT, smem, st, mc, y, none, L.ld, L.T, fm, fc, fstate_retry(ws, L), sb, segs,
                          TVArgs{});
    }

    // Time-varying model: elements from the TVElem records `el`, smoothing
    // aggregates fused as in the time-invariant scan.
    static int launch_filter_tv(void* ws, const Layout& L, const float* el, float* fm, float* fc,
                                const TVArgs& tv, cudaStream_t st) {
        constexpr int smem = filter_dyn_smem<N, FNT>();
        auto k = filter_scan_kernel<N, M, FNT, FCH, false, true, false, true, REF_DETECT, false>;
        auto kr = filter_scan_kernel<N, M, FNT, FCH, false, true, false, true, REF_FP64, true>;
        static const bool ok = allow_smem(k, smem) && allow_smem(kr, smem);
        if (!ok) return KS_ECUDA;
        const ModelConst<N, M>* mc = mconst(ws, L);
        const float* none = nullptr;
        float* sb = sblk(ws, L);
        int rc = launch_pdl(k, L.ntf, FNT, smem, st, mc, none, el, L.ld, L.T, fm, fc, fstate(ws, L), sb, no_segs(),
                            tv);
        if (rc) return rc;
        return launch_pdl(kr, L.ntf, FNT, smem, st, mc, none, el, L.ld, L.T, fm, fc, fstate_retry(ws, L), sb,
                          no_segs(), tv);
    }

    static int launch_filter_soa(void* ws, const Layout& L, const float* el, float* fm, float* fc,
                                 cudaStream_t st) {
        constexpr int smem = filter_dyn_smem<N, FNT>();
        auto k = filter_scan_kernel<N, M, FNT, FCH, false, false, false, false>;
        static const bool ok = allow_smem(k, smem);
        if (!ok) return KS_ECUDA;
        k<<<L.ntf, FNT, smem, st>>>(mconst(ws, L), nullptr, el, L.ld, L.T, fm, fc, fstate(ws, L), nullptr,
                                    no_segs(), TVArgs{});
        return launch_status();
    }

    template <bool FROM_AGG, bool SEG, bool TV = false>
    static int launch_smoother(void* ws, const Layout& L, const float* fm, const float* fc, float* sm,
                               float* sc, Segs<N, M> segs, cudaStream_t st, TVArgs tv = TVArgs{}) {
        constexpr int smem = smoother_dyn_smem<N, SNT>();
        auto k = smoother_scan_kernel<N, M, SNT, SCH, FROM_AGG, SEG, TV>;
        static const bool ok = allow_smem(k, smem);
        if (!ok) return KS_ECUDA;
        const float* sb = FROM_AGG ? sblk(ws, L) : nullptr;
        return launch_pdl(k, L.nts, SNT, smem, st, (const ModelConst<N, M>*)mconst(ws, L), (const float*)fm,
                          (const float*)fc, L.T, sm, sc, sstate(ws, L), sb, segs, tv);
    }

    static int build_elements(const ks_model* m, const float* y, int64_t T, void* ws, size_t ws_bytes,
                              cudaStream_t st) {
        const Layout L = layout(T);
        int rc = check_common(m, T, ws, ws_bytes, L.bytes_elements);
        if (rc) return rc;
        if (!y || !aligned16(y)) return KS_EINVAL;
        if ((rc = prep(m, y, ws, L, st))) return rc;
        float* el = reinterpret_cast<float*>(static_cast<char*>(ws) + L.off_elems);
        const int blocks = (int)std::min<int64_t>((T + 255) / 256, 152 * 8);
        build_elements_kernel<N, M><<<blocks, 256, 0, st>>>(mconst(ws, L), y, T, el, L.ld);
        return launch_status();
    }

    static int filter_scan(const ks_model* m, int64_t T, void* ws, size_t ws_bytes, float* fm, float* fc,
                           cudaStream_t st) {
        const Layout L = layout(T);
        int rc = check_common(m, T, ws, ws_bytes, L.bytes_elements);
        if (rc) return rc;
        if (!fm || !fc || !aligned16(fm) || !aligned16(fc)) return KS_EINVAL;
        if ((rc = reset_flags(ws, L, st))) return rc;
        const float* el = reinterpret_cast<const float*>(static_cast<char*>(ws) + L.off_elems);
        return launch_filter_soa(ws, L, el, fm, fc, st);
    }

    static int smooth_scan(const ks_model* m, int64_t T, const float* fm, const float* fc, void* ws,
                           size_t ws_bytes, float* sm, float* sc, cudaStream_t st) {
        const Layout L = layout(T);
        int rc = check_common(m, T, ws, ws_bytes, L.bytes_smooth);
        if (rc) return rc;
        if (!fm || !fc || !sm || !sc || !aligned16(fm) || !aligned16(fc) || !aligned16(sm) || !aligned16(sc))
            return KS_EINVAL;
        if ((rc = prep(m, nullptr, ws, L, st))) return rc;
        return launch_smoother<false, false>(ws, L, fm, fc, sm, sc, no_segs(), st);
    }

    static int record(void* const* ev, int i, cudaStream_t st) {
        if (!ev || !ev[i]) return KS_OK;
        return record_event(ev[i], st) == cudaSuccess ? KS_OK : KS_ECUDA;
    }

    static size_t tv_bytes(int64_t T) { return layout(T).bytes_elements; }

    // Time-varying model (m->time_varying = 1): the filtering elements are
    // materialised in their measurement form (TVElem records) from the
    // per-step arrays; the forward scan combines them with the rank-ny
    // operators and folds each thread's Lemma 5 elements, built from the next
    // step's transition, for the reverse scan.  Needs the KS_WS_ELEMENTS
    // workspace.
    static int smooth_tv(const ks_model* m, const float* y, int64_t T, void* ws, size_t ws_bytes, float* fm,
                         float* fc, float* sm, float* sc, cudaStream_t st, void* const* ev) {
        if (!m->F || !m->Q || !m->H || !m->R || !m->m0 || !m->P0) return KS_EINVAL;
        if (m->time_varying != 1) return KS_EUNSUPPORTED;
        if (!aligned16(m->F) || !aligned16(m->Q) || !aligned16(m->H) || !aligned16(m->R) ||
            (m->u && !aligned16(m->u)) || (m->d && !aligned16(m->d)))
            return KS_EINVAL;   // per-step rows are read with vector loads
        if (T < 1 || T > 0x7fffffffLL) return KS_EINVAL;
        const Layout L = layout(T);
        if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < L.bytes_elements) return KS_EINVAL;
        const bool own = (fm == nullptr) || (fc == nullptr);
        const bool filter_only = (sm == nullptr) && (sc == nullptr);
        if (!y || !aligned16(y) || (filter_only && own)) return KS_EINVAL;
        if (!filter_only && (!sm || !sc || !aligned16(sm) || !aligned16(sc))) return KS_EINVAL;
        if (own) {
            fm = reinterpret_cast<float*>(static_cast<char*>(ws) + L.off_fmean);
            fc = reinterpret_cast<float*>(static_cast<char*>(ws) + L.off_fcov);
        } else if (!aligned16(fm) || !aligned16(fc)) {
            return KS_EINVAL;
        }
        const TVArgs tv{m->F, m->u, m->Q, m->H, m->d, m->R, m->m0, m->P0};
        float* el = reinterpret_cast<float*>(static_cast<char*>(ws) + L.off_elems);
        uint32_t* z = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + L.off_flags);
        int rc;
        if ((rc = record(ev, 0, st))) return rc;
        const int blocks = (int)std::min<int64_t>((T + 255) / 256, 152 * 8);
        static_assert(TVElem<N, M>::kFloats <= NCOMP, "records fit the elements region");
        tv_elements_kernel<N, M><<<blocks, 256, 0, st>>>(tv, y, T, el, status(ws), z, (int)(L.flags_bytes / 4));
        if ((rc = launch_status())) return rc;
        if ((rc = record(ev, 1, st))) return rc;
        if ((rc = launch_filter_tv(ws, L, el, fm, fc, tv, st))) return rc;
        if ((rc = record(ev, 2, st))) return rc;
        if (!filter_only && (rc = launch_smoother<true, false, true>(ws, L, fm, fc, sm, sc, no_segs(), st, tv)))
            return rc;
        return record(ev, 3, st);
    }

    static int smooth(const ks_model* m, const float* y, int64_t T, void* ws, size_t ws_bytes, float* fm,
                      float* fc, float* sm, float* sc, cudaStream_t st, void* const* ev) {
        return smooth_v(m, y, T, ws, ws_bytes, fm, fc, sm, sc, st, ev, FCH == 32);
    }
    // `fold`: full blocks of a time-invariant model go through the linear
    // block fold (coefficients built by the preparation), else element by element.
    static int smooth_v(const ks_model* m, const float* y, int64_t T, void* ws, size_t ws_bytes, float* fm,
                        float* fc, float* sm, float* sc, cudaStream_t st, void* const* ev, bool fold) {
        if (m && m->time_varying) return smooth_tv(m, y, T, ws, ws_bytes, fm, fc, sm, sc, st, ev);
        const Layout L = layout(T);
        const bool own = (fm == nullptr) || (fc == nullptr);
        const bool filter_only = (sm == nullptr) && (sc == nullptr);
        int rc = check_common(m, T, ws, ws_bytes, own ? L.bytes_elements : L.bytes_smooth);
        if (rc) return rc;
        if (!y || !aligned16(y) || (filter_only && own)) return KS_EINVAL;
        if (!filter_only && (!sm || !sc || !aligned16(sm) || !aligned16(sc))) return KS_EINVAL;
        if (own) {
            fm = reinterpret_cast<float*>(static_cast<char*>(ws) + L.off_fmean);
            fc = reinterpret_cast<float*>(static_cast<char*>(ws) + L.off_fcov);
        } else if (!aligned16(fm) || !aligned16(fc)) {
            return KS_EINVAL;
        }
        if ((rc = record(ev, 0, st))) return rc;
        if ((rc = prep(m, y, ws, L, st, fold))) return rc;
        if ((rc = record(ev, 1, st))) return rc;
        const Segs<N, M> segs{nullptr, nullptr, 1, fold ? coef(ws, L) : nullptr};
        if ((rc = launch_filter_fused<false>(ws, L, y, fm, fc, segs, st))) return rc;
        if ((rc = record(ev, 2, st))) return rc;
        if (!filter_only && (rc = launch_smoother<true, false>(ws, L, fm, fc, sm, sc, no_segs(), st))) return rc;
        return record(ev, 3, st);
    }

    // B sequences laid end to end (offsets in mb->offsets), T steps in total.
    static int smooth_batch(const ks_model_batch* mb, const float* y, int64_t T, void* ws, size_t ws_bytes,
                            float* fm, float* fc, float* sm, float* sc, cudaStream_t st) {
        return smooth_batch_v(mb, y, T, ws, ws_bytes, fm, fc, sm, sc, st, false);
    }
    static int smooth_batch_v(const ks_model_batch* mb, const float* y, int64_t T, void* ws, size_t ws_bytes,
                              float* fm, float* fc, float* sm, float* sc, cudaStream_t st, bool fold) {
        if (!mb || !mb->F || !mb->Q || !mb->H || !mb->R || !mb->m0 || !mb->P0 || !mb->offsets)
            return KS_EINVAL;
        if (mb->B < 1 || mb->B > T || T < 1 || T > 0x7fffffffLL) return KS_EINVAL;
        const Layout L = layout(T, mb->B);
        if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < L.bytes_smooth) return KS_EINVAL;
        if (!y || !fm || !fc || !sm || !sc) return KS_EINVAL;
        if (!aligned16(y) || !aligned16(fm) || !aligned16(fc) || !aligned16(sm) || !aligned16(sc))
            return KS_EINVAL;
        uint32_t* z = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + L.off_flags);
        auto k = fold ? prep_kernel<N, M, true> : prep_kernel<N, M, false>;
        k<<<mb->B, kPrepThreads, prep_smem(), st>>>(mb->F, mb->u, mb->Q, mb->H, mb->d, mb->R, mb->m0, mb->P0, y,
                                                    mconst(ws, L), status(ws), z, (int)(L.flags_bytes / 4),
                                                    mb->offsets, T, status(ws) + HDR_FIRST_TILE,
                                                    fold ? coef(ws, L) : nullptr, FCH);
        int rc = launch_status();
        if (rc) return rc;
        const Segs<N, M> segs{mconst(ws, L), mb->offsets, mb->B, fold ? coef(ws, L) : nullptr};
        if ((rc = launch_filter_fused<true>(ws, L, y, fm, fc, segs, st))) return rc;
        return launch_smoother<true, true>(ws, L, fm, fc, sm, sc, segs, st);
    }

    static int fcomb_batch(int64_t count, const float* l, const float* r, float* o, void* ws, cudaStream_t st) {
        if (count <= 0) return KS_OK;
        const int blocks = (int)std::min<int64_t>((count + 127) / 128, 152 * 16);
        filter_combine_batch_kernel<N><<<blocks, 128, 0, st>>>(l, r, o, count, status(ws));
        return launch_status();
    }

    static int scomb_batch(int64_t count, const float* l, const float* r, float* o, void*, cudaStream_t st) {
        if (count <= 0) return KS_OK;
        const int blocks = (int)std::min<int64_t>((count + 127) / 128, 152 * 16);
        smoother_combine_batch_kernel<N><<<blocks, 128, 0, st>>>(l, r, o, count);
        return launch_status();
    }

    // ---- time-shard aggregates (ks_shard.cuh): 128 threads x 32 steps per block
    static constexpr int ANT = 128, ACH = 32;

    static Layout agg_layout(int64_t T) {
        Layout L{};
        L.T = T;
        L.B = 1;
        const int64_t nblk = (T + (int64_t)ANT * ACH - 1) / ((int64_t)ANT * ACH);
        L.ntf = L.nts = (int)nblk;
        size_t off = 256;
        L.off_const = off;
        off = align_up(off + sizeof(ModelConst<N, M>), 256);
        L.off_flags = off;
        L.flags_bytes = 16;
        off = align_up(off + L.flags_bytes, 256);
        L.off_sblk = off;                                   // one packed element per block
        off = align_up(off + 4 * (size_t)NCOMP * (size_t)nblk, 256);
        L.bytes_smooth = L.bytes_elements = off;
        return L;
    }
    static size_t agg_bytes(int64_t T) { return agg_layout(T).bytes_smooth; }

    static int faggregate(const ks_model* m, const float* y, int64_t T, int first, void* ws, size_t ws_bytes,
                          float* out, cudaStream_t st) {
        const Layout L = agg_layout(T);
        int rc = check_common(m, T, ws, ws_bytes, L.bytes_smooth);
        if (rc) return rc;
        if (!y || !out || !aligned16(y)) return KS_EINVAL;
        if ((rc = prep(m, y, ws, L, st))) return rc;
        float* blk = reinterpret_cast<float*>(static_cast<char*>(ws) + L.off_sblk);
        filter_fold_kernel<N, M, ANT, ACH><<<L.ntf, ANT, 0, st>>>(mconst(ws, L), y, T, first, blk, status(ws));
        if ((rc = launch_status())) return rc;
        fold_packed_kernel<FilterFold<N>, ANT><<<1, ANT, 0, st>>>(blk, L.ntf, out, status(ws));
        return launch_status();
    }

    static int saggregate(const ks_model* m, int64_t T, const float* fm, const float* fc, int last, void* ws,
                          size_t ws_bytes, float* out, cudaStream_t st) {
        const Layout L = agg_layout(T);
        int rc = check_common(m, T, ws, ws_bytes, L.bytes_smooth);
        if (rc) return rc;
        if (!fm || !fc || !out) return KS_EINVAL;
        if ((rc = prep(m, nullptr, ws, L, st))) return rc;
        float* blk = reinterpret_cast<float*>(static_cast<char*>(ws) + L.off_sblk);
        smoother_fold_kernel<N, M, ANT, ACH><<<L.nts, ANT, 0, st>>>(mconst(ws, L), fm, fc, T, last, blk,
                                                                     status(ws));
        if ((rc = launch_status())) return rc;
        fold_packed_kernel<SmootherFold<N>, ANT><<<1, ANT, 0, st>>>(blk, L.nts, out, status(ws));
        return launch_status();
    }

    static constexpr VTable vtable() {
        return VTable{N, M, &layout, &build_elements, &filter_scan, &smooth_scan, &smooth, &smooth_batch,
                      &fcomb_batch, &scomb_batch, &agg_bytes, &faggregate, &saggregate, &tv_bytes};
    }
    static constexpr ChunkVariant chunk_variant() { return ChunkVariant{&layout, &smooth_v, &smooth_batch_v}; }
};

// Steps per thread of the fused smooth / smooth_batch scans, picked from
// {4, 8, 16, 32} by the total number of steps T.  A block scan covers
// 128 * chunk steps, so short inputs need short chunks to launch enough
// blocks for the 152 SMs; long inputs keep 32 steps per thread, which cuts
// the per-block look-back, aggregate and per-thread-prefix work per step.
// The built-in crossovers are where the measured times of neighbouring chunk
// lengths cross for nx = 2, 4 and 6 on GB300 (single sequences and
// segmented batches alike); ks_set_chunk_rules replaces them per state size
// with a table measured by the tuner.
inline int builtin_chunk_index(int64_t T) {
    return T < 96 * 1024 ? 0 : T < 192 * 1024 ? 1 : T < 640 * 1024 ? 2 : 3;
}

// Whether the built-in table folds full blocks with the linear block fold:
// single-size calls with 32 steps per thread (where the per-call coefficient
// build is small against the scans), not the mixed-size launch.
inline bool builtin_fold(int nx, int64_t T) { return nx != 0 && builtin_chunk_index(T) == 3; }

// Choice for a call over T steps of state size nx (2, 4 or 6; 0: mixed-size
// batches), from the table set by ks_set_chunk_rules, else the built-in one
// (ks_api.cu): bits 0-1 the chunk index (0..3 for 4, 8, 16, 32 steps per
// thread), bit 2 the block-fold flag.
int chunk_choice(int nx, int64_t T);
inline int chunk_index_for(int nx, int64_t T) { return chunk_choice(nx, T) & 3; }

// Per-(nx, ny) table of the four chunk variants; each instantiation file
// defines it (the 4-, 8- and 16-step variants compile in their own units).
template <int N, int M>
struct ChunkTable {
    static const ChunkVariant* const v[4];
};

// The registered function table: every entry of the 32-step Impl, except that
// smooth and smooth_batch go to the chunk variant chosen by T, and the
// workspace sizes cover every variant (offsets stay the 32-step layout's,
// which the element-building and scan-only entry points use).
template <int N, int M>
struct Tuned {
    using Base = Impl<N, M, 32>;
    static Layout layout(int64_t T, int B) {
        Layout L = Base::layout(T, B);
        for (int i = 0; i < 4; ++i) {
            const Layout Li = ChunkTable<N, M>::v[i]->layout(T, B);
            L.bytes_smooth = std::max(L.bytes_smooth, Li.bytes_smooth);
            L.bytes_elements = std::max(L.bytes_elements, Li.bytes_elements);
        }
        return L;
    }
    static int smooth(const ks_model* m, const float* y, int64_t T, void* ws, size_t ws_bytes, float* fm,
                      float* fc, float* sm, float* sc, cudaStream_t st, void* const* ev) {
        const int c = chunk_choice(N, T);
        return ChunkTable<N, M>::v[c & 3]->smooth(m, y, T, ws, ws_bytes, fm, fc, sm, sc, st, ev, (c & 4) != 0);
    }
    static int smooth_batch(const ks_model_batch* mb, const float* y, int64_t T, void* ws, size_t ws_bytes,
                            float* fm, float* fc, float* sm, float* sc, cudaStream_t st) {
        // segmented batches fold element by element: every sequence would need its
        // own coefficients, read from L2 in phase 1 (measured slower in the
        // mixed-size launch)
        return ChunkTable<N, M>::v[chunk_index_for(N, T)]->smooth_batch(mb, y, T, ws, ws_bytes, fm, fc, sm, sc, st,
                                                                         false);
    }
    static size_t tv_bytes(int64_t T) { return layout(T, 1).bytes_elements; }
    static constexpr VTable vtable() {
        VTable t = Base::vtable();
        t.layout = &layout;
        t.tv_bytes = &tv_bytes;
        t.smooth = &smooth;
        t.smooth_batch = &smooth_batch;
        return t;
    }
};

// Registry (one entry per compiled (nx, ny)).
const VTable* find_impl(int nx, int ny);

}  // namespace ks
