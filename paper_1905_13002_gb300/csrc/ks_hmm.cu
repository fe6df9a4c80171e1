// ks_hmm.cu -- C ABI of the discrete-state (HMM) filter and smoother
// (ks_hmm.cuh): workspace layout, argument checks and launches.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/ks.h"
#include "ks_hmm.cuh"
#include "ks_hmmw.cuh"
#include "ks_impl.cuh"

namespace ks {
namespace hmm {
namespace {

struct HLayout {
    int64_t T = 0;
    int ntiles = 0;
    int64_t nblk = 0;
    size_t off_const = 0, off_flags = 0, flags_bytes = 0;
    size_t off_fagg = 0, off_fpre = 0, off_sagg = 0, off_spre = 0, off_sblk = 0, bytes = 0;
};

// K states, CH steps per thread, 128 threads per block.
template <int K, int CH>
struct HImpl {
    static constexpr int NT = 128;
    static constexpr int64_t TILE = (int64_t)NT * CH;

    static HLayout layout(int64_t T) {
        HLayout L;
        L.T = T;
        L.ntiles = (int)((T + TILE - 1) / TILE);
        L.nblk = (T + CH - 1) / CH;
        size_t off = 256;                                   // status word + reserved
        L.off_const = off;
        off = align_up(off + sizeof(Const<K>), 256);
        L.off_flags = off;                                  // [fcounter, scounter, 2 pad][fflags][sflags]
        L.flags_bytes = 16 + 4 * 2 * (size_t)L.ntiles;
        off = align_up(off + L.flags_bytes, 256);
        L.off_fagg = off;
        off = align_up(off + sizeof(FE<K>) * (size_t)L.ntiles, 256);
        L.off_fpre = off;
        off = align_up(off + sizeof(FS<K>) * (size_t)L.ntiles, 256);
        L.off_sagg = off;
        off = align_up(off + sizeof(SE<K>) * (size_t)L.ntiles, 256);
        L.off_spre = off;
        off = align_up(off + sizeof(SS<K>) * (size_t)L.ntiles, 256);
        L.off_sblk = off;                                   // one smoothing aggregate per CH steps
        off = align_up(off + sizeof(SE<K>) * (size_t)L.nblk, 256);
        L.bytes = off;
        return L;
    }

    static ScanState state(void* ws, const HLayout& L, bool forward) {
        char* b = static_cast<char*>(ws);
        ScanState s;
        s.counter = reinterpret_cast<uint32_t*>(b + L.off_flags + (forward ? 0 : 4));
        s.flags = reinterpret_cast<uint32_t*>(b + L.off_flags + 16 + (forward ? 0 : 4 * (size_t)L.ntiles));
        s.agg = reinterpret_cast<float*>(b + (forward ? L.off_fagg : L.off_sagg));
        s.pre = reinterpret_cast<float*>(b + (forward ? L.off_fpre : L.off_spre));
        s.status = static_cast<uint32_t*>(ws);
        s.spin_limit = kSpinLimit;
        return s;
    }

    static int smooth(const ks_hmm* h, const float* lik, int64_t T, void* ws, size_t ws_bytes, float* filt,
                      float* smooth, float* loglik, cudaStream_t st, void* const* ev) {
        const HLayout L = layout(T);
        if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < L.bytes) return KS_EINVAL;
        char* b = static_cast<char*>(ws);
        const Const<K>* cg = reinterpret_cast<const Const<K>*>(b + L.off_const);
        float* sblk = reinterpret_cast<float*>(b + L.off_sblk);
        auto rec = [&](int i) {
            return (ev && ev[i] && record_event(ev[i], st) != cudaSuccess) ? KS_ECUDA
                                                                                                        : KS_OK;
        };
        int rc;
        if ((rc = rec(0))) return rc;
        hmm_prep_kernel<K><<<1, 64, 0, st>>>(h->pi, h->Pi, reinterpret_cast<Const<K>*>(b + L.off_const),
                                             static_cast<uint32_t*>(ws),
                                             reinterpret_cast<uint32_t*>(b + L.off_flags), (int)(L.flags_bytes / 4));
        if ((rc = launch_status())) return rc;
        if ((rc = rec(1))) return rc;
        hmm_filter_kernel<K, NT, CH><<<L.ntiles, NT, 0, st>>>(cg, lik, T, filt, loglik, state(ws, L, true), sblk);
        if ((rc = launch_status())) return rc;
        if ((rc = rec(2))) return rc;
        if (smooth) {
            hmm_smoother_kernel<K, NT, CH><<<L.ntiles, NT, 0, st>>>(cg, filt, T, smooth, state(ws, L, false), sblk);
            if ((rc = launch_status())) return rc;
        }
        return rec(3);
    }
};

// Steps per thread by length: short inputs take 4 (more blocks for the
// SMs), longer ones 16 and then 32 (fewer tiles, so less block-scan work per
// step).  At K = 8 and T = 2^20, 32 steps per thread take 0.32 ms against
// 0.38 ms at 16 and 0.49 ms at 8.
constexpr int64_t kMidT = 256 * 1024, kLongT = 768 * 1024;

template <int K>
size_t bytes(int64_t T) {
    return std::max({HImpl<K, 4>::layout(T).bytes, HImpl<K, 16>::layout(T).bytes, HImpl<K, 32>::layout(T).bytes});
}

template <int K>
int run(const ks_hmm* h, const float* lik, int64_t T, void* ws, size_t ws_bytes, float* filt, float* smooth,
        float* loglik, cudaStream_t st, void* const* ev) {
    if (T < kMidT) return HImpl<K, 4>::smooth(h, lik, T, ws, ws_bytes, filt, smooth, loglik, st, ev);
    if (T < kLongT) return HImpl<K, 16>::smooth(h, lik, T, ws, ws_bytes, filt, smooth, loglik, st, ev);
    return HImpl<K, 32>::smooth(h, lik, T, ws, ws_bytes, filt, smooth, loglik, st, ev);
}

// K = 16, 32: one K-lane group per chain of CH steps, NG chains per tile
// (ks_hmmw.cuh).
template <int K>
struct WImpl {
    static constexpr int NW = 4, CH = 64, NWS = 4;
    static constexpr int NG = NW * 32 / K;
    struct WLayout {
        int64_t nch = 0;
        int ntiles = 0;
        size_t off_const = 0, off_fexcl = 0, off_fsp0 = 0, off_fsp1 = 0, off_schain = 0, off_sexcl = 0,
               off_ssp0 = 0, off_ssp1 = 0, bytes = 0;
    };
    static WLayout layout(int64_t T) {
        using D = hmmw::Dims<K>;
        WLayout L;
        L.nch = (T + CH - 1) / CH;
        L.ntiles = (int)((L.nch + NG - 1) / NG);
        size_t off = 256;
        L.off_const = off;
        off = align_up(off + sizeof(hmmw::Const<K>), 256);
        L.off_fexcl = off;
        off = align_up(off + 4 * (size_t)D::FREC * L.nch, 256);
        L.off_fsp0 = off;
        off = align_up(off + 4 * (size_t)D::FREC * L.ntiles, 256);
        L.off_fsp1 = off;
        off = align_up(off + 4 * (size_t)D::FREC * L.ntiles, 256);
        L.off_schain = off;
        off = align_up(off + 4 * (size_t)D::SREC * L.nch, 256);
        L.off_sexcl = off;
        off = align_up(off + 4 * (size_t)D::SREC * L.nch, 256);
        L.off_ssp0 = off;
        off = align_up(off + 4 * (size_t)D::SREC * L.ntiles, 256);
        L.off_ssp1 = off;
        off = align_up(off + 4 * (size_t)D::SREC * L.ntiles, 256);
        L.bytes = off;
        return L;
    }

    static int smooth(const ks_hmm* h, const float* lik, int64_t T, void* ws, size_t ws_bytes, float* filt,
                      float* smooth, float* loglik, cudaStream_t st, void* const* ev) {
        using namespace hmmw;
        const WLayout L = layout(T);
        const int sgrid_tiles = NWS * 32 / K;   // tiles per spine block
        if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < L.bytes) return KS_EINVAL;
        if (!aligned16(lik)) return KS_EINVAL;   // likelihood rows are read as float4
        char* b = static_cast<char*>(ws);
        uint32_t* stat = static_cast<uint32_t*>(ws);
        hmmw::Const<K>* cg = reinterpret_cast<hmmw::Const<K>*>(b + L.off_const);
        hmmw::Bufs bf;
        bf.fexcl = reinterpret_cast<float*>(b + L.off_fexcl);
        bf.fspine0 = reinterpret_cast<float*>(b + L.off_fsp0);
        bf.fspine1 = reinterpret_cast<float*>(b + L.off_fsp1);
        bf.schain = reinterpret_cast<float*>(b + L.off_schain);
        bf.sexcl = reinterpret_cast<float*>(b + L.off_sexcl);
        bf.sspine0 = reinterpret_cast<float*>(b + L.off_ssp0);
        bf.sspine1 = reinterpret_cast<float*>(b + L.off_ssp1);
        auto rec = [&](int i) {
            return (ev && ev[i] && record_event(ev[i], st) != cudaSuccess) ? KS_ECUDA
                                                                                                        : KS_OK;
        };
        const int sgrid = (L.ntiles + sgrid_tiles - 1) / sgrid_tiles;
        int rc;
        if ((rc = rec(0))) return rc;
        hmmw::prep_kernel<K><<<1, 64, 0, st>>>(h->pi, h->Pi, cg, stat);
        if ((rc = launch_status())) return rc;
        if ((rc = rec(1))) return rc;
        filter_reduce_kernel<K, NW, CH><<<L.ntiles, NW * 32, 0, st>>>(cg, lik, T, bf, stat);
        if ((rc = launch_status())) return rc;
        const float* src = bf.fspine0;
        float* dst = bf.fspine1;
        for (int s = 1; s < L.ntiles; s <<= 1) {
            spine_kernel<true, K, NWS><<<sgrid, NWS * 32, 0, st>>>(src, dst, L.ntiles, s, stat);
            if ((rc = launch_status())) return rc;
            float* t = const_cast<float*>(src);
            src = dst;
            dst = t;
        }
        filter_apply_kernel<K, NW, CH><<<L.ntiles, NW * 32, 0, st>>>(cg, lik, T, filt, loglik, bf, src, stat);
        if ((rc = launch_status())) return rc;
        if ((rc = rec(2))) return rc;
        if (smooth) {
            smoother_reduce_kernel<K, NW><<<L.ntiles, NW * 32, 0, st>>>(L.nch, bf, stat);
            if ((rc = launch_status())) return rc;
            const float* ssrc = bf.sspine0;
            float* sdst = bf.sspine1;
            for (int s = 1; s < L.ntiles; s <<= 1) {
                spine_kernel<false, K, NWS><<<sgrid, NWS * 32, 0, st>>>(ssrc, sdst, L.ntiles, s, stat);
                if ((rc = launch_status())) return rc;
                float* t = const_cast<float*>(ssrc);
                ssrc = sdst;
                sdst = t;
            }
            smoother_apply_kernel<K, NW, CH><<<L.ntiles, NW * 32, 0, st>>>(cg, filt, T, smooth, bf, ssrc, stat);
            if ((rc = launch_status())) return rc;
        }
        return rec(3);
    }
};

}  // namespace
}  // namespace hmm
}  // namespace ks

using namespace ks;

extern "C" {

int ks_hmm_supported(int K) { return (K == 2 || K == 4 || K == 8 || K == 16 || K == 32) ? 1 : 0; }

size_t ks_hmm_workspace_bytes(int K, int64_t T) {
    if (T < 1 || T > 0x7fffffffLL) return 0;
    switch (K) {
        case 2: return hmm::bytes<2>(T);
        case 4: return hmm::bytes<4>(T);
        case 8: return hmm::bytes<8>(T);
        case 16: return hmm::WImpl<16>::layout(T).bytes;
        case 32: return hmm::WImpl<32>::layout(T).bytes;
        default: return 0;
    }
}

int ks_hmm_smooth_traced(const ks_hmm* h, const float* lik, int64_t T, void* ws, size_t ws_bytes, float* filt,
                         float* smooth, float* loglik, void* stream, void* const* events) {
    if (!h || !h->pi || !h->Pi) return KS_EINVAL;
    if (!ks_hmm_supported(h->K)) return KS_EUNSUPPORTED;
    if (T < 1 || T > 0x7fffffffLL || !lik || !filt) return KS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (h->K) {
        case 2: return hmm::run<2>(h, lik, T, ws, ws_bytes, filt, smooth, loglik, st, events);
        case 4: return hmm::run<4>(h, lik, T, ws, ws_bytes, filt, smooth, loglik, st, events);
        case 8: return hmm::run<8>(h, lik, T, ws, ws_bytes, filt, smooth, loglik, st, events);
        case 16: return hmm::WImpl<16>::smooth(h, lik, T, ws, ws_bytes, filt, smooth, loglik, st, events);
        default: return hmm::WImpl<32>::smooth(h, lik, T, ws, ws_bytes, filt, smooth, loglik, st, events);
    }
}

int ks_hmm_smooth(const ks_hmm* h, const float* lik, int64_t T, void* ws, size_t ws_bytes, float* filt,
                  float* smooth, float* loglik, void* stream) {
    return ks_hmm_smooth_traced(h, lik, T, ws, ws_bytes, filt, smooth, loglik, stream, nullptr);
}

}  // extern "C"
