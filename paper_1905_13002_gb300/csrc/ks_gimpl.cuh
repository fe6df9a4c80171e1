// ks_gimpl.cuh -- host side of the one-warp-per-chain instantiations (larger
// nx): workspace layout and launches (reduce, spine levels, apply per scan)
// behind the same C ABI as ks_impl.cuh.
#pragma once

#include "ks_gscan.cuh"
#include "ks_impl.cuh"

namespace ks {

template <int N, int M, int NW, int CH>
struct GImpl {
    static constexpr int FS = grp::Dim<N>::FSLOT, SS = grp::Dim<N>::SSLOT;
    using SM = grp::GSmem<N, M, NW>;
    static constexpr int NG = SM::NG;                      // chains per tile (one lane group each)
    static constexpr int64_t TILE = (int64_t)NG * CH;

    static size_t prep_smem() { return sizeof(PrepSmem<N, M>) + sizeof(ModelConst<N, M>) + 16; }

    static Layout layout(int64_t T, int B = 1) {
        Layout L;
        L.T = T;
        L.B = B;
        L.ld = 0;
        const int64_t nch = (T + CH - 1) / CH;
        L.ntf = L.nts = (int)((nch + NG - 1) / NG);
        size_t off = 256;
        L.off_const = off;
        off = align_up(off + sizeof(ModelConst<N, M>) * (size_t)B, 256);
        L.off_flags = off;                                  // zeroed by the preparation kernel
        L.flags_bytes = 16;
        off = align_up(off + L.flags_bytes, 256);
        L.off_fagg = off;                                   // filter: two spine buffers
        off = align_up(off + 4 * (size_t)FS * L.ntf * 2, 256);
        L.off_fpre = off;                                   // filter chains
        off = align_up(off + 4 * (size_t)FS * (size_t)L.ntf * NG * 2, 256);
        L.off_sagg = off;                                   // smoother: two spine buffers
        off = align_up(off + 4 * (size_t)SS * L.nts * 2, 256);
        L.off_spre = off;                                   // smoother chains
        off = align_up(off + 4 * (size_t)SS * (size_t)L.nts * NG * 2, 256);
        L.off_sblk = off;                                   // smoothing elements, one slot per step
        off = align_up(off + 4 * (size_t)SS * (size_t)T, 256);
        L.bytes_smooth = off;
        L.off_elems = off;
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
    static uint32_t* status(void* ws) { return static_cast<uint32_t*>(ws); }

    static void buffers(void* ws, const Layout& L, grp::GBuf& fb, grp::GBuf& sb) {
        char* b = static_cast<char*>(ws);
        float* fa = reinterpret_cast<float*>(b + L.off_fagg);
        fb.spine0 = fa;
        fb.spine1 = fa + (size_t)FS * L.ntf;
        fb.chains = reinterpret_cast<float*>(b + L.off_fpre);
        float* sa = reinterpret_cast<float*>(b + L.off_sagg);
        sb.spine0 = sa;
        sb.spine1 = sa + (size_t)SS * L.nts;
        sb.chains = reinterpret_cast<float*>(b + L.off_spre);
        fb.elems = nullptr;
        sb.elems = reinterpret_cast<float*>(b + L.off_sblk);
    }

    template <class K>
    static bool allow_smem(K kernel, int bytes) {
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
    }

    static int prep(const float* F, const float* u, const float* Q, const float* H, const float* d,
                    const float* R, const double* m0, const double* P0, const float* y, int B,
                    const int64_t* off, void* ws, const Layout& L, cudaStream_t st) {
        const int smem = (int)prep_smem();
        auto k = prep_kernel<N, M>;
        static const bool ok = allow_smem(k, smem);
        if (!ok) return KS_ECUDA;
        uint32_t* z = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + L.off_flags);
        k<<<B, kPrepThreads, smem, st>>>(F, u, Q, H, d, R, m0, P0, y, mconst(ws, L), status(ws), z,
                                (int)(L.flags_bytes / 4), off, L.T, nullptr, nullptr, 0);
        return launch_status();
    }

    // Per scan: a reduce launch, log2(tiles) spine launches, an apply launch.
    template <bool SEG, bool TV = false>
    static int scans(void* ws, const Layout& L, const float* y, float* fm, float* fc, float* sm, float* sc,
                     Segs<N, M> segs, cudaStream_t st, void* const* ev, bool filter, bool smoother) {
        grp::GBuf fb, sb;
        buffers(ws, L, fb, sb);
        constexpr int smem = SM::BYTES;
        constexpr int SW = grp::gspine_warps<N>();
        constexpr int ssmem = grp::GSpineSmem<N, SW>::BYTES;
        constexpr int SG = grp::GSpineSmem<N, SW>::NG;          // tiles per spine block
        uint32_t* stat = status(ws);
        int rc;
        if (filter) {
            auto kr = grp::gfilter_reduce_kernel<N, M, NW, CH, SEG, TV>;
            auto ks = grp::gspine_filter_kernel<N, SW>;
            auto ka = grp::gfilter_apply_kernel<N, M, NW, CH, SEG, TV>;
            static const bool ok = allow_smem(kr, smem) && allow_smem(ks, ssmem) && allow_smem(ka, smem);
            if (!ok) return KS_ECUDA;
            kr<<<L.ntf, NW * 32, smem, st>>>(mconst(ws, L), y, L.T, fb, stat, segs);
            if ((rc = launch_status())) return rc;
            const float* src = fb.spine0;
            float* dst = fb.spine1;
            for (int s = 1; s < L.ntf; s <<= 1) {
                ks<<<(L.ntf + SG - 1) / SG, SW * 32, ssmem, st>>>(src, dst, L.ntf, s, stat);
                if ((rc = launch_status())) return rc;
                float* t = const_cast<float*>(src);
                src = dst;
                dst = t;
            }
            ka<<<L.ntf, NW * 32, smem, st>>>(mconst(ws, L), y, L.T, fm, fc, fb, src, stat, segs);
            if ((rc = launch_status())) return rc;
        }
        if (ev && ev[2] && record_event(ev[2], st) != cudaSuccess) return KS_ECUDA;
        if (smoother) {
            auto kr = grp::gsmoother_reduce_kernel<N, M, NW, CH, SEG, TV>;
            auto ks = grp::gspine_smoother_kernel<N, SW>;
            auto ka = grp::gsmoother_apply_kernel<N, M, NW, CH>;
            static const bool ok = allow_smem(kr, smem) && allow_smem(ks, ssmem) && allow_smem(ka, smem);
            if (!ok) return KS_ECUDA;
            kr<<<L.nts, NW * 32, smem, st>>>(mconst(ws, L), fm, fc, L.T, sb, stat, segs);
            if ((rc = launch_status())) return rc;
            const float* src = sb.spine0;
            float* dst = sb.spine1;
            for (int s = 1; s < L.nts; s <<= 1) {
                ks<<<(L.nts + SG - 1) / SG, SW * 32, ssmem, st>>>(src, dst, L.nts, s, stat);
                if ((rc = launch_status())) return rc;
                float* t = const_cast<float*>(src);
                src = dst;
                dst = t;
            }
            ka<<<L.nts, NW * 32, smem, st>>>(L.T, sm, sc, sb, src, stat);
            if ((rc = launch_status())) return rc;
        }
        return KS_OK;
    }

    static int check(const ks_model* m, int64_t T, void* ws, size_t ws_bytes, size_t need) {
        if (!m || !m->F || !m->Q || !m->H || !m->R || !m->m0 || !m->P0) return KS_EINVAL;
        if (m->time_varying != 0) return KS_EUNSUPPORTED;
        if (T < 1 || T > 0x7fffffffLL) return KS_EINVAL;
        if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < need) return KS_EINVAL;
        return KS_OK;
    }

    static int build_elements(const ks_model*, const float*, int64_t, void*, size_t, cudaStream_t) {
        return KS_EUNSUPPORTED;   // materialised elements are offered for the register-resident sizes
    }
    static int filter_scan(const ks_model*, int64_t, void*, size_t, float*, float*, cudaStream_t) {
        return KS_EUNSUPPORTED;
    }

    static int smooth_scan(const ks_model* m, int64_t T, const float* fm, const float* fc, void* ws,
                           size_t ws_bytes, float* sm, float* sc, cudaStream_t st) {
        const Layout L = layout(T);
        int rc = check(m, T, ws, ws_bytes, L.bytes_smooth);
        if (rc) return rc;
        if (!fm || !fc || !sm || !sc) return KS_EINVAL;
        if ((rc = prep(m->F, m->u, m->Q, m->H, m->d, m->R, m->m0, m->P0, nullptr, 1, nullptr, ws, L, st)))
            return rc;
        return scans<false>(ws, L, nullptr, const_cast<float*>(fm), const_cast<float*>(fc), sm, sc,
                            Segs<N, M>{nullptr, nullptr, 1}, st, nullptr, false, true);
    }

    // Time-varying model: per-step constants (prep_kernel for step 0 with its
    // FP64 k = 1 element, tv_const_kernel for the rest) after the elements
    // region, read by the scans through a per-step Cursor.
    static size_t tv_offset(int64_t T) { return align_up(layout(T).bytes_elements, 256); }
    static size_t tv_bytes(int64_t T) { return tv_offset(T) + sizeof(ModelConst<N, M>) * (size_t)T; }

    static int smooth_tv(const ks_model* m, const float* y, int64_t T, void* ws, size_t ws_bytes, float* fm,
                         float* fc, float* sm, float* sc, cudaStream_t st, void* const* ev) {
        if (!m->F || !m->Q || !m->H || !m->R || !m->m0 || !m->P0) return KS_EINVAL;
        if (m->time_varying != 1) return KS_EUNSUPPORTED;
        if (T < 1 || T > 0x7fffffffLL) return KS_EINVAL;
        if (!aligned16(m->F) || !aligned16(m->Q) || !aligned16(m->H) || !aligned16(m->R) ||
            (m->u && !aligned16(m->u)) || (m->d && !aligned16(m->d)))
            return KS_EINVAL;
        const Layout L = layout(T);
        if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < tv_bytes(T)) return KS_EINVAL;
        const bool own = (fm == nullptr) || (fc == nullptr);
        const bool filter_only = (sm == nullptr) && (sc == nullptr);
        if (!y || (filter_only && own) || (!filter_only && (!sm || !sc))) return KS_EINVAL;
        if (own) {
            fm = reinterpret_cast<float*>(static_cast<char*>(ws) + L.off_fmean);
            fc = reinterpret_cast<float*>(static_cast<char*>(ws) + L.off_fcov);
        }
        auto* tvc = reinterpret_cast<ModelConst<N, M>*>(static_cast<char*>(ws) + tv_offset(T));
        const TVArgs tv{m->F, m->u, m->Q, m->H, m->d, m->R, m->m0, m->P0};
        int rc;
        if (ev && ev[0] && record_event(ev[0], st) != cudaSuccess) return KS_ECUDA;
        {
            const int smem = (int)prep_smem();
            auto k = prep_kernel<N, M>;
            static const bool ok = allow_smem(k, smem);
            if (!ok) return KS_ECUDA;
            uint32_t* z = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + L.off_flags);
            k<<<1, kPrepThreads, smem, st>>>(m->F, m->u, m->Q, m->H, m->d, m->R, m->m0, m->P0, y, tvc, status(ws), z,
                                             (int)(L.flags_bytes / 4), nullptr, T, nullptr, nullptr, 0);
            if ((rc = launch_status())) return rc;
        }
        if (T > 1) {
            const int blocks = (int)std::min<int64_t>((T + 127) / 128, 152 * 8);
            tv_const_kernel<N, M><<<blocks, 128, 0, st>>>(tv, T, tvc, status(ws));
            if ((rc = launch_status())) return rc;
        }
        if (ev && ev[1] && record_event(ev[1], st) != cudaSuccess) return KS_ECUDA;
        if ((rc = scans<false, true>(ws, L, y, fm, fc, sm, sc, Segs<N, M>{tvc, nullptr, 1}, st, ev, true,
                                     !filter_only)))
            return rc;
        if (ev && ev[3] && record_event(ev[3], st) != cudaSuccess) return KS_ECUDA;
        return KS_OK;
    }

    static int smooth(const ks_model* m, const float* y, int64_t T, void* ws, size_t ws_bytes, float* fm,
                      float* fc, float* sm, float* sc, cudaStream_t st, void* const* ev) {
        if (m && m->time_varying) return smooth_tv(m, y, T, ws, ws_bytes, fm, fc, sm, sc, st, ev);
        const Layout L = layout(T);
        const bool own = (fm == nullptr) || (fc == nullptr);
        const bool filter_only = (sm == nullptr) && (sc == nullptr);
        int rc = check(m, T, ws, ws_bytes, own ? L.bytes_elements : L.bytes_smooth);
        if (rc) return rc;
        if (!y || (filter_only && own) || (!filter_only && (!sm || !sc))) return KS_EINVAL;
        if (own) {
            fm = reinterpret_cast<float*>(static_cast<char*>(ws) + L.off_fmean);
            fc = reinterpret_cast<float*>(static_cast<char*>(ws) + L.off_fcov);
        }
        if (ev && ev[0] && record_event(ev[0], st) != cudaSuccess) return KS_ECUDA;
        if ((rc = prep(m->F, m->u, m->Q, m->H, m->d, m->R, m->m0, m->P0, y, 1, nullptr, ws, L, st))) return rc;
        if (ev && ev[1] && record_event(ev[1], st) != cudaSuccess) return KS_ECUDA;
        if ((rc = scans<false>(ws, L, y, fm, fc, sm, sc, Segs<N, M>{nullptr, nullptr, 1}, st, ev, true,
                               !filter_only)))
            return rc;
        if (ev && ev[3] && record_event(ev[3], st) != cudaSuccess) return KS_ECUDA;
        return KS_OK;
    }

    static int smooth_batch(const ks_model_batch* mb, const float* y, int64_t T, void* ws, size_t ws_bytes,
                            float* fm, float* fc, float* sm, float* sc, cudaStream_t st) {
        if (!mb || !mb->F || !mb->Q || !mb->H || !mb->R || !mb->m0 || !mb->P0 || !mb->offsets)
            return KS_EINVAL;
        if (mb->B < 1 || mb->B > T || T < 1 || T > 0x7fffffffLL) return KS_EINVAL;
        const Layout L = layout(T, mb->B);
        if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < L.bytes_smooth) return KS_EINVAL;
        if (!y || !fm || !fc || !sm || !sc) return KS_EINVAL;
        int rc = prep(mb->F, mb->u, mb->Q, mb->H, mb->d, mb->R, mb->m0, mb->P0, y, mb->B, mb->offsets, ws, L, st);
        if (rc) return rc;
        return scans<true>(ws, L, y, fm, fc, sm, sc, Segs<N, M>{mconst(ws, L), mb->offsets, mb->B}, st, nullptr,
                           true, true);
    }

    static int no_comb(int64_t, const float*, const float*, float*, void*, cudaStream_t) { return KS_EUNSUPPORTED; }
    static size_t no_agg_bytes(int64_t) { return 0; }
    static int no_fagg(const ks_model*, const float*, int64_t, int, void*, size_t, float*, cudaStream_t) {
        return KS_EUNSUPPORTED;
    }
    static int no_sagg(const ks_model*, int64_t, const float*, const float*, int, void*, size_t, float*,
                       cudaStream_t) {
        return KS_EUNSUPPORTED;
    }

    static constexpr VTable vtable() {
        return VTable{N, M, &layout, &build_elements, &filter_scan, &smooth_scan, &smooth, &smooth_batch,
                      &no_comb, &no_comb, &no_agg_bytes, &no_fagg, &no_sagg, &tv_bytes};
    }
};

}  // namespace ks
