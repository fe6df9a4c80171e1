// ks_timpl.cuh -- host side of the nx = 32 tensor-core scans: workspace
// layout and launches behind the same C ABI as ks_impl.cuh: per scan a
// reduce launch, log2(tiles) spine launches and an apply launch.  Segmented
// batches at this size run on the CUDA-core group kernels (ks_gimpl.cuh).
#pragma once

#include "ks_gimpl.cuh"
#include "ks_tscan.cuh"

namespace ks {

template <int N, int M, int NW, int CH>
struct TImpl {
    static constexpr int FR = tc::Rec<N>::F, SR = tc::Rec<N>::S;
    using FSM = tc::TSmem<N, M, NW, tc::FConst<N, M>>;
    using SSM = tc::TSmem<N, M, NW, tc::SConst<N, M>>;

    static Layout layout(int64_t T) {
        Layout L;
        L.T = T;
        L.B = 1;
        L.ld = 0;
        const int64_t nch = (T + CH - 1) / CH;
        L.ntf = L.nts = (int)((nch + NW - 1) / NW);
        const size_t nchp = (size_t)L.ntf * NW;
        size_t off = 256;
        L.off_const = off;
        off = align_up(off + sizeof(ModelConst<N, M>), 256);
        L.off_flags = off;                                  // zeroed by the preparation kernel
        L.flags_bytes = 16;
        off = align_up(off + L.flags_bytes, 256);
        L.off_fagg = off;                                   // filter: two spine buffers
        off = align_up(off + 4 * (size_t)FR * L.ntf * 2, 256);
        L.off_fpre = off;                                   // filter chains
        off = align_up(off + 4 * (size_t)FR * nchp * 2, 256);
        L.off_sagg = off;                                   // smoother: two spine buffers
        off = align_up(off + 4 * (size_t)SR * L.nts * 2, 256);
        L.off_spre = off;                                   // smoother chains
        off = align_up(off + 4 * (size_t)SR * nchp * 2, 256);
        L.off_sblk = off;                                   // smoothing elements, one per step
        off = align_up(off + 4 * (size_t)SR * (size_t)T, 256);
        L.bytes_smooth = off;
        L.off_elems = off;
        L.off_fmean = off;
        off = align_up(off + 4 * (size_t)N * (size_t)T, 256);
        L.off_fcov = off;
        off = align_up(off + 4 * (size_t)N * N * (size_t)T, 256);
        L.bytes_elements = off;
        return L;
    }

    static void buffers(void* ws, const Layout& L, tc::TBuf& fb, tc::TBuf& sb) {
        char* b = static_cast<char*>(ws);
        float* fs = reinterpret_cast<float*>(b + L.off_fagg);
        fb.spine0 = fs;
        fb.spine1 = fs + (size_t)FR * L.ntf;
        fb.chains = reinterpret_cast<float*>(b + L.off_fpre);
        fb.elems = nullptr;
        float* ss = reinterpret_cast<float*>(b + L.off_sagg);
        sb.spine0 = ss;
        sb.spine1 = ss + (size_t)SR * L.nts;
        sb.chains = reinterpret_cast<float*>(b + L.off_spre);
        sb.elems = reinterpret_cast<float*>(b + L.off_sblk);
    }

    template <class K>
    static bool allow_smem(K kernel, int bytes) {
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
    }

    static int scans(void* ws, const Layout& L, const float* y, float* fm, float* fc, float* sm, float* sc,
                     cudaStream_t st, void* const* ev, bool filter, bool smoother) {
        using FSP = tc::SpineSmem<N, tc::kSpineWarps, tc::kSpineBufF>;
        using SSP = tc::SpineSmem<N, tc::kSpineWarps, tc::kSpineBufS>;
        constexpr int SW = tc::kSpineWarps;
        tc::TBuf fb, sb;
        buffers(ws, L, fb, sb);
        uint32_t* status = static_cast<uint32_t*>(ws);
        const ModelConst<N, M>* mc =
            reinterpret_cast<const ModelConst<N, M>*>(static_cast<char*>(ws) + L.off_const);
        int rc;
        if (filter) {
            auto kr = tc::tfilter_reduce_kernel<N, M, NW, CH>;
            auto ks = tc::tspine_filter_kernel<N, SW>;
            auto ka = tc::tfilter_apply_kernel<N, M, NW, CH>;
            static const bool ok = allow_smem(kr, (int)sizeof(FSM)) && allow_smem(ks, (int)sizeof(FSP)) &&
                                   allow_smem(ka, (int)sizeof(FSM));
            if (!ok) return KS_ECUDA;
            kr<<<L.ntf, NW * 32, sizeof(FSM), st>>>(mc, y, L.T, fb, status);
            if ((rc = launch_status())) return rc;
            const float* src = fb.spine0;
            float* dst = fb.spine1;
            for (int s = 1; s < L.ntf; s <<= 1) {
                ks<<<(L.ntf + SW - 1) / SW, SW * 32, sizeof(FSP), st>>>(src, dst, L.ntf, s, status);
                if ((rc = launch_status())) return rc;
                float* t = const_cast<float*>(src);
                src = dst;
                dst = t;
            }
            ka<<<L.ntf, NW * 32, sizeof(FSM), st>>>(mc, y, L.T, fm, fc, fb, src, status);
            if ((rc = launch_status())) return rc;
        }
        if (ev && ev[2] && record_event(ev[2], st) != cudaSuccess) return KS_ECUDA;
        if (smoother) {
            auto kr = tc::tsmoother_reduce_kernel<N, M, NW, CH>;
            auto ks = tc::tspine_smoother_kernel<N, SW>;
            auto ka = tc::tsmoother_apply_kernel<N, M, NW, CH>;
            static const bool ok = allow_smem(kr, (int)sizeof(SSM)) && allow_smem(ks, (int)sizeof(SSP)) &&
                                   allow_smem(ka, (int)sizeof(SSM));
            if (!ok) return KS_ECUDA;
            kr<<<L.nts, NW * 32, sizeof(SSM), st>>>(mc, fm, fc, L.T, sb, status);
            if ((rc = launch_status())) return rc;
            const float* src = sb.spine0;
            float* dst = sb.spine1;
            for (int s = 1; s < L.nts; s <<= 1) {
                ks<<<(L.nts + SW - 1) / SW, SW * 32, sizeof(SSP), st>>>(src, dst, L.nts, s, status);
                if ((rc = launch_status())) return rc;
                float* t = const_cast<float*>(src);
                src = dst;
                dst = t;
            }
            ka<<<L.nts, NW * 32, sizeof(SSM), st>>>(L.T, sm, sc, sb, src, status);
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

    // The caller's posterior buffers are moved with 16-byte vector accesses.
    static bool vec_ok(const float* a, const float* b, const float* c, const float* d) {
        return aligned16(a) && aligned16(b) && aligned16(c) && aligned16(d);
    }

    static int smooth_scan(const ks_model* m, int64_t T, const float* fm, const float* fc, void* ws,
                           size_t ws_bytes, float* sm, float* sc, cudaStream_t st) {
        const Layout L = layout(T);
        int rc = check(m, T, ws, ws_bytes, L.bytes_smooth);
        if (rc) return rc;
        if (!fm || !fc || !sm || !sc) return KS_EINVAL;
        if (!vec_ok(fm, fc, sm, sc)) return KS_EINVAL;
        if ((rc = GImpl<N, M, NW, CH>::prep(m->F, m->u, m->Q, m->H, m->d, m->R, m->m0, m->P0, nullptr, 1,
                                            nullptr, ws, L, st)))
            return rc;
        return scans(ws, L, nullptr, const_cast<float*>(fm), const_cast<float*>(fc), sm, sc, st, nullptr, false,
                     true);
    }

    static int smooth(const ks_model* m, const float* y, int64_t T, void* ws, size_t ws_bytes, float* fm,
                      float* fc, float* sm, float* sc, cudaStream_t st, void* const* ev) {
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
        if (!vec_ok(fm, fc, filter_only ? fm : sm, filter_only ? fc : sc)) return KS_EINVAL;
        if (ev && ev[0] && record_event(ev[0], st) != cudaSuccess) return KS_ECUDA;
        if ((rc = GImpl<N, M, NW, CH>::prep(m->F, m->u, m->Q, m->H, m->d, m->R, m->m0, m->P0, y, 1, nullptr, ws,
                                            L, st)))
            return rc;
        if (ev && ev[1] && record_event(ev[1], st) != cudaSuccess) return KS_ECUDA;
        if ((rc = scans(ws, L, y, fm, fc, sm, sc, st, ev, true, !filter_only))) return rc;
        if (ev && ev[3] && record_event(ev[3], st) != cudaSuccess) return KS_ECUDA;
        return KS_OK;
    }
};

}  // namespace ks
