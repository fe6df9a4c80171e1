// ks_mixed.cuh -- one preparation, one forward and one reverse launch over a
// batch whose sequences have different state sizes (nx in {2, 4, 6}).
//
// The sequences come in up to three groups, one per state size, each laid
// out as a segmented batch of its own (sequences end to end, per-sequence
// model constants, a CSR offset table; the resets of Section III-C's
// block-level elements keep every combine inside its sequence).  Each scan
// is one launch whose thread blocks take work items -- (group, tile) pairs --
// from one atomic counter, nx = 6 tiles first, then nx = 4, then nx = 2, so
// the heaviest work starts first and the lighter tiles fill the tail.  A
// block runs the scan body specialised for its item's state size (the same
// bodies as the single-size kernels of ks_scan.cuh); its look-back only
// reads tiles of its own group, which were claimed earlier from the same
// counter and so belong to running or finished blocks.
#pragma once

#include "ks_impl.cuh"

namespace ks {

template <class X>
constexpr X cmax(X a, X b) { return a > b ? a : b; }

// One group: its sequences' model arrays (prep), its segmented axis, its
// data and its part of the workspace.
template <int N, int M>
struct MixedGroup {
    int B = 0;            // sequences (0: the group is absent)
    int ntiles = 0;       // forward tiles = reverse tiles
    int64_t T = 0;        // steps
    const float *F = nullptr, *u = nullptr, *Q = nullptr, *H = nullptr, *d = nullptr, *R = nullptr;
    const double *m0 = nullptr, *P0 = nullptr;
    Segs<N, M> segs{nullptr, nullptr, 0};   // constants [B] (written by prep), offsets [B + 1]
    const float* y = nullptr;
    float *fmean = nullptr, *fcov = nullptr, *smean = nullptr, *scov = nullptr;
    ScanState fs{}, ss{};   // look-back flags and records of the two scans (counters unused)
    ScanState fs2{};        // the forward scan's retry with refinement
    float* sagg = nullptr;  // fused smoothing aggregates, one per forward block
    uint32_t* zero = nullptr;   // the group's flags region
    int nzero = 0;
    int ch = 0;                 // steps per thread of the launch (block-fold coefficients)
};

using MG6 = MixedGroup<6, 3>;
using MG4 = MixedGroup<4, 2>;
using MG2 = MixedGroup<2, 1>;

// Work-queue counters of the two scans and the status word.
struct MixedQueue {
    uint32_t* fcounter;
    uint32_t* scounter;
    uint32_t* fcounter2;   // the forward scan's retry
    uint32_t* status;
};

constexpr int kMixedThreads = 128;

template <int N, int M, bool FOLD>
KS_DEV void mixed_prep_one(char* dsm, int sg, const MixedGroup<N, M>& g) {
    prep_body<N, M, FOLD>(dsm, sg, g.B, g.F, g.u, g.Q, g.H, g.d, g.R, g.m0, g.P0, g.y,
                    const_cast<ModelConst<N, M>*>(g.segs.mcg), g.fs.status, g.zero, g.nzero, g.segs.off, g.T,
                    nullptr, const_cast<BlockCoef<N, M>*>(g.segs.coef), g.ch);
}

// One block per sequence of all groups (nx = 6 sequences first); block 0 also
// zeroes the two work-queue counters.  (CH only makes one copy per
// instantiation unit; FOLD: build the block-fold coefficients.)
template <int CH, bool FOLD>
__global__ void __launch_bounds__(kPrepThreads) mixed_prep_kernel(MG6 g6, MG4 g4, MG2 g2, MixedQueue q) {
    extern __shared__ __align__(16) char prep_dsm[];
    int b = (int)blockIdx.x;
    if (b == 0 && threadIdx.x == 0) {
        *q.fcounter = 0u;
        *q.scounter = 0u;
        *q.fcounter2 = 0u;
    }
    if (b < g6.B) { mixed_prep_one<6, 3, FOLD>(prep_dsm, b, g6); return; }
    b -= g6.B;
    if (b < g4.B) { mixed_prep_one<4, 2, FOLD>(prep_dsm, b, g4); return; }
    b -= g4.B;
    if (b < g2.B) mixed_prep_one<2, 1, FOLD>(prep_dsm, b, g2);
}

template <int N, int M>
constexpr size_t mixed_prep_smem_of() { return prep_dyn_smem<N, M>(); }
constexpr size_t mixed_prep_smem() {
    return cmax(cmax(mixed_prep_smem_of<6, 3>(), mixed_prep_smem_of<4, 2>()), mixed_prep_smem_of<2, 1>());
}

template <int CH, int REF, bool RETRY>
KS_DEV void mixed_filter_tile(const MG6& g6, const MG4& g4, const MG2& g2, const MixedQueue& q);

// REF / RETRY as for filter_scan_kernel: the first launch detects
// ill-conditioned inverses, the retry repeats the scan with refinement only
// when the first met one.
template <int CH, int REF, bool RETRY>
__global__ void __launch_bounds__(kMixedThreads) mixed_filter_kernel(MG6 g6, MG4 g4, MG2 g2, MixedQueue q) {
    pdl_wait();
    if constexpr (RETRY) {
        if (*(volatile uint32_t*)(q.status + HDR_NEED) == 0u) {
            pdl_trigger();
            return;
        }
    }
    mixed_filter_tile<CH, REF, RETRY>(g6, g4, g2, q);
    pdl_trigger();
}

// Dynamic shared memory of one size's body: its block-scan state first, its
// staging buffers after it.  A block carves the layout of its item's size out
// of one dynamic allocation sized for the largest, so that the big block-scan
// state of nx = 6 and the staging buffers of nx = 4 never add up.
__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) / 16 * 16; }
template <int N, int M>
constexpr size_t mixed_filter_smem_of() {
    return align16(sizeof(FilterSmem<N, M, kMixedThreads>)) + (size_t)filter_dyn_smem<N, kMixedThreads>();
}
template <int N, int M>
constexpr size_t mixed_smoother_smem_of() {
    return align16(sizeof(SmootherSmem<N, M, kMixedThreads>)) + (size_t)smoother_dyn_smem<N, kMixedThreads>();
}
constexpr int mixed_filter_smem() {
    return (int)cmax(cmax(mixed_filter_smem_of<6, 3>(), mixed_filter_smem_of<4, 2>()), mixed_filter_smem_of<2, 1>());
}
constexpr int mixed_smoother_smem() {
    return (int)cmax(cmax(mixed_smoother_smem_of<6, 3>(), mixed_smoother_smem_of<4, 2>()),
                     mixed_smoother_smem_of<2, 1>());
}

template <int N, int M, int CH, int REF, bool RETRY>
KS_DEV void mixed_filter_one(char* dsm, int t, const MixedGroup<N, M>& g) {
    auto& sm = *reinterpret_cast<FilterSmem<N, M, kMixedThreads>*>(dsm);
    char* stage = dsm + align16(sizeof(FilterSmem<N, M, kMixedThreads>));
    filter_scan_body<N, M, kMixedThreads, CH, true, true, true, false, REF>(
        sm, stage, t, g.y, nullptr, 0, g.T, g.fmean, g.fcov, RETRY ? g.fs2 : g.fs, g.sagg, g.segs, TVArgs{});
}

template <int CH, int REF, bool RETRY>
KS_DEV void mixed_filter_tile(const MG6& g6, const MG4& g4, const MG2& g2, const MixedQueue& q) {
    __shared__ int s_tile;
    extern __shared__ __align__(16) char dsm[];
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(RETRY ? q.fcounter2 : q.fcounter, 1u);
    __syncthreads();
    int t = s_tile;
    if (t < g6.ntiles) {
        mixed_filter_one<6, 3, CH, REF, RETRY>(dsm, t, g6);
    } else if ((t -= g6.ntiles) < g4.ntiles) {
        mixed_filter_one<4, 2, CH, REF, RETRY>(dsm, t, g4);
    } else if ((t -= g4.ntiles) < g2.ntiles) {
        mixed_filter_one<2, 1, CH, REF, RETRY>(dsm, t, g2);
    }
}

template <int N, int M, int CH>
KS_DEV void mixed_smoother_one(char* dsm, int t, const MixedGroup<N, M>& g) {
    auto& sm = *reinterpret_cast<SmootherSmem<N, M, kMixedThreads>*>(dsm);
    char* stage = dsm + align16(sizeof(SmootherSmem<N, M, kMixedThreads>));
    if constexpr (Stage<N>::kOn) {   // this thread's two staging mbarriers
        mbar_init(&sm.mbars[2 * threadIdx.x], 1);
        mbar_init(&sm.mbars[2 * threadIdx.x + 1], 1);
        fence_proxy_async();
        __syncthreads();
    }
    smoother_scan_body<N, M, kMixedThreads, CH, true, true, false>(sm, stage, t, g.fmean, g.fcov, g.T, g.smean,
                                                                   g.scov, g.ss, g.sagg, g.segs, TVArgs{});
}

template <int CH>
__global__ void __launch_bounds__(kMixedThreads, kRevMinBlocks<4>) mixed_smoother_kernel(MG6 g6, MG4 g4, MG2 g2,
                                                                                       MixedQueue q) {
    __shared__ int s_tile;
    extern __shared__ __align__(16) char dsm[];
    pdl_wait();
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(q.scounter, 1u);
    __syncthreads();
    int t = s_tile;
    if (t < g6.ntiles) {
        mixed_smoother_one<6, 3, CH>(dsm, t, g6);
    } else if ((t -= g6.ntiles) < g4.ntiles) {
        mixed_smoother_one<4, 2, CH>(dsm, t, g4);
    } else if ((t -= g4.ntiles) < g2.ntiles) {
        mixed_smoother_one<2, 1, CH>(dsm, t, g2);
    }
    pdl_trigger();
}

// ---------------------------------------------------------------- host side
// Workspace: the 256-byte header (status word, refinement counter, wait
// settings), 256 bytes of work-queue counters, then one region per present
// group (nx = 6, 4, 2), each laid out as that size's segmented workspace.
constexpr size_t kMixedQueueOff = 256;
constexpr size_t kMixedGroupsOff = 512;

template <int CH>
struct Mixed {
    template <int N, int M>
    static Layout layout_of(const ks_batch_group& g) {
        return Impl<N, M, CH>::layout(g.total_T, g.models.B);
    }

    // Byte offset of each size's region (index 0: nx = 6, 1: nx = 4, 2: nx = 2)
    // for groups[slot[i]] (slot -1: absent); returns the total size.
    static size_t regions(const ks_batch_group* gs, const int (&slot)[3], size_t (&base)[3]) {
        size_t off = kMixedGroupsOff;
        for (int i = 0; i < 3; ++i) {
            base[i] = off;
            if (slot[i] < 0) continue;
            const ks_batch_group& g = gs[slot[i]];
            const Layout L = i == 0 ? layout_of<6, 3>(g) : i == 1 ? layout_of<4, 2>(g) : layout_of<2, 1>(g);
            off = align_up(off + L.bytes_smooth, 256);
        }
        return off;
    }

    template <int N, int M>
    static MixedGroup<N, M> group(const ks_batch_group* gs, int slot, char* ws, size_t base, bool fold) {
        MixedGroup<N, M> o;
        if (slot < 0) return o;
        const ks_batch_group& g = gs[slot];
        const ks_model_batch& mb = g.models;
        const Layout L = Impl<N, M, CH>::layout(g.total_T, mb.B);
        char* b = ws + base;
        o.B = mb.B;
        o.ntiles = L.ntf;
        o.T = g.total_T;
        o.F = mb.F; o.u = mb.u; o.Q = mb.Q; o.H = mb.H; o.d = mb.d; o.R = mb.R;
        o.m0 = mb.m0; o.P0 = mb.P0;
        o.segs = Segs<N, M>{reinterpret_cast<const ModelConst<N, M>*>(b + L.off_const), mb.offsets, mb.B,
                            fold ? reinterpret_cast<const BlockCoef<N, M>*>(b + L.off_coef) : nullptr};
        o.ch = fold ? CH : 0;
        o.y = g.y;
        o.fmean = g.fmean; o.fcov = g.fcov; o.smean = g.smean; o.scov = g.scov;
        uint32_t* status = reinterpret_cast<uint32_t*>(ws);
        o.fs.counter = nullptr;
        o.fs.flags = reinterpret_cast<uint32_t*>(b + L.off_flags + 16);
        o.fs.agg = reinterpret_cast<float*>(b + L.off_fagg);
        o.fs.pre = reinterpret_cast<float*>(b + L.off_fpre);
        o.fs.status = status;
        o.fs.spin_limit = kSpinLimit;
        o.fs2 = o.fs;
        o.fs2.flags = reinterpret_cast<uint32_t*>(b + L.off_flags + 16 + 4 * (size_t)(L.ntf + L.nts));
        o.ss.counter = nullptr;
        o.ss.flags = reinterpret_cast<uint32_t*>(b + L.off_flags + 16 + 4 * (size_t)L.ntf);
        o.ss.agg = reinterpret_cast<float*>(b + L.off_sagg);
        o.ss.pre = reinterpret_cast<float*>(b + L.off_spre);
        o.ss.status = status;
        o.ss.spin_limit = kSpinLimit;
        o.sagg = reinterpret_cast<float*>(b + L.off_sblk);
        o.zero = reinterpret_cast<uint32_t*>(b + L.off_flags);
        o.nzero = (int)(L.flags_bytes / 4);
        return o;
    }

    template <class K>
    static bool allow_smem(K kernel, int bytes) {
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess;
    }

    static int run(const ks_batch_group* gs, const int (&slot)[3], void* ws, size_t ws_bytes, cudaStream_t st,
                   bool fold) {
        size_t base[3];
        if (regions(gs, slot, base) > ws_bytes) return KS_EINVAL;
        char* w = static_cast<char*>(ws);
        const MG6 g6 = group<6, 3>(gs, slot[0], w, base[0], fold);
        const MG4 g4 = group<4, 2>(gs, slot[1], w, base[1], fold);
        const MG2 g2 = group<2, 1>(gs, slot[2], w, base[2], fold);
        const MixedQueue q{reinterpret_cast<uint32_t*>(w + kMixedQueueOff),
                           reinterpret_cast<uint32_t*>(w + kMixedQueueOff + 4),
                           reinterpret_cast<uint32_t*>(w + kMixedQueueOff + 8), reinterpret_cast<uint32_t*>(w)};
        const int nseq = g6.B + g4.B + g2.B;
        const int ntiles = g6.ntiles + g4.ntiles + g2.ntiles;
        static const bool ok = allow_smem(mixed_prep_kernel<CH, true>, (int)mixed_prep_smem()) &&
                               allow_smem(mixed_prep_kernel<CH, false>, (int)mixed_prep_smem()) &&
                               allow_smem(mixed_filter_kernel<CH, REF_DETECT, false>, mixed_filter_smem()) &&
                               allow_smem(mixed_filter_kernel<CH, REF_FP64, true>, mixed_filter_smem()) &&
                               allow_smem(mixed_smoother_kernel<CH>, mixed_smoother_smem());
        if (!ok) return KS_ECUDA;
        if (fold)
            mixed_prep_kernel<CH, true><<<nseq, kPrepThreads, mixed_prep_smem(), st>>>(g6, g4, g2, q);
        else
            mixed_prep_kernel<CH, false><<<nseq, kPrepThreads, mixed_prep_smem(), st>>>(g6, g4, g2, q);
        int rc = launch_status();
        if (rc) return rc;
        if ((rc = launch_pdl(mixed_filter_kernel<CH, REF_DETECT, false>, ntiles, kMixedThreads, mixed_filter_smem(),
                             st, g6, g4, g2, q)))
            return rc;
        if ((rc = launch_pdl(mixed_filter_kernel<CH, REF_FP64, true>, ntiles, kMixedThreads, mixed_filter_smem(), st,
                             g6, g4, g2, q)))
            return rc;
        return launch_pdl(mixed_smoother_kernel<CH>, ntiles, kMixedThreads, mixed_smoother_smem(), st, g6, g4, g2, q);
    }
};

// Per-chunk-length entry points (ks_mixed{4,8,16,32}.cu).
struct MixedVariant {
    size_t (*regions)(const ks_batch_group*, const int (&)[3], size_t (&)[3]);
    int (*run)(const ks_batch_group*, const int (&)[3], void*, size_t, cudaStream_t, bool fold);
};
template <int CH>
constexpr MixedVariant mixed_variant() { return MixedVariant{&Mixed<CH>::regions, &Mixed<CH>::run}; }

}  // namespace ks
