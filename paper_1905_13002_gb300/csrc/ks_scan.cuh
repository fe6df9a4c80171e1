// ks_scan.cuh -- the forward filtering scan, the reverse smoothing scan, the
// model-preparation and element-building kernels.
//
// Scan structure (block-level elements of Section III-C, all-prefix-sums of
// Section II-B):
//   phase 1  each thread folds CH consecutive steps into one block element;
//   phase 2  an inclusive warp scan of the block elements (shuffles), an
//            exclusive scan of the warp totals, and a decoupled look-back
//            over earlier tiles (tile = NT threads x CH steps) that yields the
//            prefix entering this tile;
//   phase 3  each thread starts from the prefix entering its block (a
//            filtered / smoothed posterior, since every full prefix of the
//            filter has A = 0 and every full suffix of the smoother has
//            E = 0) and applies its CH elements one at a time, writing one
//            posterior per step.
// Tiles are numbered by an atomic counter in the order thread blocks start,
// so a tile only ever waits for tiles whose blocks are already running.
// Every wait is bounded; a wait that runs out records ST_TIMEOUT in the
// status word and the kernel finishes with a zero prefix instead of hanging.
#pragma once

#include "ks_async.cuh"
#include "ks_ops.cuh"

namespace ks {

// Record a timing event on `st` (host); inside a stream capture as an
// external event node, so that every replay of the graph records it.
inline cudaError_t record_event(void* ev, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return cudaErrorUnknown;
    cudaEvent_t e = static_cast<cudaEvent_t>(ev);
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal)
                                               : cudaEventRecord(e, st);
}

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kFlagAgg = 1u;   // tile aggregate published
constexpr uint32_t kFlagPre = 2u;   // inclusive prefix published

struct ScanState {
    uint32_t* counter;   // tile counter (zeroed before launch)
    uint32_t* flags;     // per-tile flags (zeroed before launch)
    float* agg;          // per-tile aggregates
    float* pre;          // per-tile inclusive prefixes
    uint32_t* status;    // device status word (workspace header, see below)
    uint32_t spin_limit; // look-back polls before giving up (~1 s)
};

KS_DEV uint32_t wait_limit(const ScanState& ss) {
    const uint32_t o = ss.status[HDR_WAIT];
    return o != 0u ? o : ss.spin_limit;
}

template <class T>
KS_DEV T shfl_up_t(const T& x, int d) {
    static_assert(sizeof(T) % 4 == 0, "float payload");
    T y;
    const float* px = reinterpret_cast<const float*>(&x);
    float* py = reinterpret_cast<float*>(&y);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) py[i] = __shfl_up_sync(kFull, px[i], d);
    return y;
}

template <class T>
KS_DEV T shfl_down_t(const T& x, int d) {
    T y;
    const float* px = reinterpret_cast<const float*>(&x);
    float* py = reinterpret_cast<float*>(&y);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) py[i] = __shfl_down_sync(kFull, px[i], d);
    return y;
}

template <class T>
KS_DEV T shfl_t(const T& x, int src) {
    T y;
    const float* px = reinterpret_cast<const float*>(&x);
    float* py = reinterpret_cast<float*>(&y);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) py[i] = __shfl_sync(kFull, px[i], src);
    return y;
}

template <class T>
KS_DEV void store_plain(float* dst, const T& x) {
    const float* px = reinterpret_cast<const float*>(&x);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) dst[i] = px[i];
}

// Loads of data published by other thread blocks go through L2 (.cg).
template <class T>
KS_DEV T load_cg(const float* src) {
    T y;
    float* py = reinterpret_cast<float*>(&y);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) py[i] = __ldcg(src + i);
    return y;
}

KS_DEV uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

KS_DEV void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Poll a flag until it is non-zero, at most `limit` times with a growing
// sleep; returns 0 if it never became non-zero.
KS_DEV uint32_t wait_flag(const uint32_t* p, uint32_t limit) {
    uint32_t v = ld_acquire(p);
    uint32_t ns = 32;
    for (uint32_t it = 0; v == 0u; ++it) {
        if (it >= limit) return 0u;
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
        v = ld_acquire(p);
    }
    return v;
}

// ---------------------------------------------------------------- vector I/O
template <int N>
KS_DEV void load_row(const float* __restrict__ p, float (&v)[N]) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N; i += 4) {
            float4 t = __ldg(reinterpret_cast<const float4*>(p + i));
            v[i] = t.x; v[i + 1] = t.y; v[i + 2] = t.z; v[i + 3] = t.w;
        }
    } else if constexpr (N % 2 == 0) {
#pragma unroll
        for (int i = 0; i < N; i += 2) {
            float2 t = __ldg(reinterpret_cast<const float2*>(p + i));
            v[i] = t.x; v[i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = __ldg(p + i);
    }
}

template <int N>
KS_DEV void store_row(float* __restrict__ p, const float (&v)[N]) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N; i += 4)
            *reinterpret_cast<float4*>(p + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else if constexpr (N % 2 == 0) {
#pragma unroll
        for (int i = 0; i < N; i += 2) *reinterpret_cast<float2*>(p + i) = make_float2(v[i], v[i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) p[i] = v[i];
    }
}

// Write one posterior (mean [N], covariance [N][N] from its lower triangle).
template <int N>
KS_DEV void store_posterior(float* __restrict__ mean, float* __restrict__ cov, int64_t k,
                            const float (&m)[N], const float (&S)[sym_size(N)]) {
    store_row<N>(mean + k * N, m);
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float row[N];
#pragma unroll
        for (int b = 0; b < N; ++b) row[b] = S[sidx(a, b)];
        store_row<N>(cov + (k * N + a) * N, row);
    }
}

template <int N>
KS_DEV void load_posterior(const float* __restrict__ mean, const float* __restrict__ cov, int64_t k,
                           float (&m)[N], float (&S)[sym_size(N)]) {
    load_row<N>(mean + k * N, m);
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float row[N];
        load_row<N>(cov + (k * N + a) * N, row);
#pragma unroll
        for (int b = 0; b <= a; ++b) S[sidx(a, b)] = row[b];
    }
}

template <int N>
KS_DEV float finite_probe(const float (&m)[N], const float (&S)[sym_size(N)]) {
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < N; ++a) s += m[a] + S[sidx(a, a)];
    return s;
}

template <int M>
KS_DEV void load_meas(const float* __restrict__ y, int64_t k, float (&v)[M]) {
    load_row<M>(y + k * M, v);
}

// Element k of the materialised structure-of-arrays layout.
template <int N>
KS_DEV FElem<N> load_soa(const float* __restrict__ el, int64_t ld, int64_t k) {
    FElem<N> e;
    constexpr int oA = 0, ob = N * N, oC = N * N + N, oe = 2 * N * N + N, oJ = 2 * N * N + 2 * N;
#pragma unroll
    for (int a = 0; a < N * N; ++a) e.A[a] = __ldg(el + (oA + a) * ld + k);
#pragma unroll
    for (int a = 0; a < N; ++a) {
        e.b[a] = __ldg(el + (ob + a) * ld + k);
        e.eta[a] = __ldg(el + (oe + a) * ld + k);
    }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            e.C[sidx(a, b)] = __ldg(el + (oC + a * N + b) * ld + k);
            e.J[sidx(a, b)] = __ldg(el + (oJ + a * N + b) * ld + k);
        }
    return e;
}

template <int N, int M>
KS_DEV void load_coef(const BlockCoef<N, M>* __restrict__ g, BlockCoef<N, M>& s, int tid, int nt) {
    static_assert(sizeof(BlockCoef<N, M>) % 16 == 0, "vector copy");
    const float4* src = reinterpret_cast<const float4*>(g);
    float4* dst = reinterpret_cast<float4*>(&s);
    for (int i = tid; i < (int)(sizeof(BlockCoef<N, M>) / 16); i += nt) dst[i] = src[i];
}

template <int N, int M>
KS_DEV void load_const(const ModelConst<N, M>* __restrict__ g, ModelConst<N, M>& s, int tid, int nt) {
    const float* src = reinterpret_cast<const float*>(g);
    float* dst = reinterpret_cast<float*>(&s);
    for (int i = tid; i < (int)(sizeof(ModelConst<N, M>) / 4); i += nt) dst[i] = __ldg(src + i);
}

// ---------------------------------------------------------------- segments
// Scans may run over several independent sequences laid end to end (segment
// s = steps [off[s], off[s+1]) of the concatenated axis).  No combine needs
// to know where a segment starts: a segment's first filtering element has
// A_1 = 0 (Lemma 3), so any prefix combined with it yields exactly that
// segment's own (b_1, C_1), and its last smoothing element has E_n = 0
// (Lemma 5), so any suffix combined after it is discarded.  Only the element
// builders need each step's segment (its model constants, whether the step
// is a segment's first or last).  A single sequence is the case off = {0, T}
// with its constants in shared memory.
template <int N, int M>
struct Segs {
    const ModelConst<N, M>* mcg;   // per-segment constants [B] (batched)
    const int64_t* off;            // [B+1] (batched), else nullptr
    int B;
    const BlockCoef<N, M>* coef = nullptr;   // block-fold coefficients per segment (null: none)
};

// With TV the constants are per step (g.mcg[k] for step k of one sequence of
// g.mcg's length): the step's filtering element reads g.mcg[k], and its
// Lemma 5 element the next step's transition, g.mcg[k + 1] (trans(k)).
template <int N, int M, bool SEG, bool TV = false>
struct Cursor {
    static_assert(!(SEG && TV), "a time-varying model is one sequence");
    const ModelConst<N, M>* mc;
    const ModelConst<N, M>* base;
    int64_t start, end;
    int s;

    KS_DEV void seek(const Segs<N, M>& g, const ModelConst<N, M>* single, int64_t k, int64_t T) {
        if constexpr (TV) {
            base = g.mcg;
            mc = base + k;
            start = 0;
            end = T;
            s = 0;
        } else if constexpr (!SEG) {
            mc = single;
            start = 0;
            end = T;
            s = 0;
        } else {
            int lo = 0, hi = g.B - 1;          // largest s with off[s] <= k
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(g.off + mid) <= k) lo = mid;
                else hi = mid - 1;
            }
            s = lo;
            start = __ldg(g.off + s);
            end = __ldg(g.off + s + 1);
            mc = g.mcg + s;
        }
    }
    // The loops stop at the table's ends, so an inconsistent table (reported
    // by the preparation kernel) cannot take a cursor out of bounds.
    KS_DEV void forward(const Segs<N, M>& g, int64_t k) {
        if constexpr (TV) {
            mc = base + k;
        } else if constexpr (SEG) {
            while (k >= end && s < g.B - 1) {
                ++s;
                start = end;
                end = __ldg(g.off + s + 1);
                mc = g.mcg + s;
            }
        }
    }
    KS_DEV void backward(const Segs<N, M>& g, int64_t k) {
        if constexpr (TV) {
            mc = base + k;
        } else if constexpr (SEG) {
            while (k < start && s > 0) {
                --s;
                end = start;
                start = __ldg(g.off + s);
                mc = g.mcg + s;
            }
        }
    }
    KS_DEV bool first(int64_t k) const { return k == start; }
    KS_DEV bool last(int64_t k) const { return k == end - 1; }
    // Constants holding the transition that Lemma 5 reads at step k.
    KS_DEV const ModelConst<N, M>* trans(int64_t k) const {
        if constexpr (TV) return (k + 1 < end) ? base + k + 1 : mc;
        else return mc;
    }
};

// ---------------------------------------------------------------- time-varying models
// Per-step model arrays of one time-varying sequence (device, row-major FP32,
// each 16-byte aligned): F [T][N][N], u [T][N] or null, Q [T][N][N],
// H [T][M][N], d [T][M] or null, R [T][M][M]; m0 [N], P0 [N][N] FP64.  Step k is predicted from step k - 1
// with F[k], u[k], Q[k] (F[0] maps the prior N(m0, P0) to step 0) and observed
// through H[k], d[k], R[k] (the model of Section II with its indices shifted
// to start at 0).
struct TVArgs {
    const float *F, *u, *Q, *H, *d, *R;
    const double *m0, *P0;
};

// COUNT consecutive floats of step k of a step-major array whose base is
// 16-byte aligned: float4 loads when a step's block is a multiple of 16
// bytes, float2 when of 8, scalar otherwise.
template <int COUNT>
KS_DEV void load_step(const float* __restrict__ base, int64_t k, float* __restrict__ dst) {
    const float* p = base + k * COUNT;
    if constexpr (COUNT % 4 == 0) {
#pragma unroll
        for (int i = 0; i < COUNT / 4; ++i) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(p) + i);
            dst[4 * i] = q.x;
            dst[4 * i + 1] = q.y;
            dst[4 * i + 2] = q.z;
            dst[4 * i + 3] = q.w;
        }
    } else if constexpr (COUNT % 2 == 0) {
#pragma unroll
        for (int i = 0; i < COUNT / 2; ++i) {
            const float2 q = __ldg(reinterpret_cast<const float2*>(p) + i);
            dst[2 * i] = q.x;
            dst[2 * i + 1] = q.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < COUNT; ++i) dst[i] = __ldg(p + i);
    }
}

// One step's transition (what the Lemma 5 element of the step before reads).
template <int N>
struct Trans {
    float F[N * N];
    float u[N];
    float Q[sym_size(N)];
};

template <int N>
KS_DEV void load_trans(const TVArgs& tv, int64_t k, Trans<N>& t) {
    float Q[N * N];
    load_step<N * N>(tv.F, k, t.F);
    load_step<N * N>(tv.Q, k, Q);
    if (tv.u) load_step<N>(tv.u, k, t.u);
    else {
#pragma unroll
        for (int a = 0; a < N; ++a) t.u[a] = 0.f;
    }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) t.Q[sidx(a, b)] = 0.5f * (Q[a * N + b] + Q[b * N + a]);
}

// Lemma 5 element of step k of a time-varying sequence of T steps: the
// transition into step k + 1 is that step's (F, u, Q).
template <int N, int M>
KS_DEV void build_selem_tv(const TVArgs& tv, int64_t k, int64_t T, const float (&xb)[N],
                           const float (&P)[sym_size(N)], SElem<N>& e, Flags& bad) {
    if (k == T - 1) {   // Lemma 5, k = n: E = 0, g = xbar_n, L = P_n
#pragma unroll
        for (int a = 0; a < N * N; ++a) e.E[a] = 0.f;
#pragma unroll
        for (int a = 0; a < N; ++a) e.g[a] = xb[a];
#pragma unroll
        for (int a = 0; a < sym_size(N); ++a) e.L[a] = P[a];
    } else {
        Trans<N> t;
        load_trans<N>(tv, k + 1, t);
        smoother_element<N, M>(t, xb, P, e, bad);
    }
}

// Lemma 5 element of step k with no branch around its arithmetic, so that
// two calls can be interleaved: the element is always built from the step's
// transition (a time-varying model's k + 1, or k itself when k = n, whose
// result is discarded) and the k = n case (E = 0, g = xbar_n, L = P_n) then
// replaces it.
template <int N, int M, bool TV>
KS_DEV void build_selem_flat(const ModelConst<N, M>* mc, const TVArgs& tv, int64_t k, int64_t T, bool last,
                             const float (&xb)[N], const float (&P)[sym_size(N)], SElem<N>& e, Flags& bad) {
    bool b = false;
    if constexpr (TV) {
        Trans<N> t;
        load_trans<N>(tv, last ? k : k + 1, t);
        smoother_element<N, M>(t, xb, P, e, b);
    } else {
        smoother_element<N, M>(*mc, xb, P, e, b);
    }
    bad |= (b && !last) ? FL_BAD : 0u;
    if (last) {
#pragma unroll
        for (int a = 0; a < N * N; ++a) e.E[a] = 0.f;
#pragma unroll
        for (int a = 0; a < N; ++a) e.g[a] = xb[a];
#pragma unroll
        for (int a = 0; a < sym_size(N); ++a) e.L[a] = P[a];
    }
}

// ---------------------------------------------------------------- prep
// Model constants, one thread block.  k > 1 quantities in FP32 (Lemma 3 with
// the Cholesky factor of S); the k = 1 element (Kalman prediction and update
// from N(m0, P0), Lemma 3) in FP64.  Every matrix product is spread over a
// warp, one output entry per lane.  Block s
// prepares segment s (batched: the model arrays hold one model per segment
// and `off` gives the segments' first steps); block 0 also zeroes the scans'
// tile counters and flags and checks the segment table.
template <int N, int M>
struct PrepSmem {
    float F[N][N], Q[N][N], H[M][N], R[M][M], u[N], d[M], y[M];
    double m0[N], P0[N][N];
    // warp 0: the FP32 model constants
    float HQ[M][N], HF[M][N], S[M][M], Lsi[M][M], tmp[M][N], K[N][M];
    // warps 1-3: the k = 1 element in FP64 (inputs widened once, S1^{-1}, S1^{-1} H P-)
    double mm[N], FP[N][N], Pm[N][N], HP[M][N], S1[M][M], z[M];
    double dF[N][N], dQ[N][N], dH[M][N], dR[M][M], du[N], v[M], Si[M][M], W[M][N];
    int ok0, ok1;
};

constexpr int kPrepThreads = 128;   // warp 0: FP32 constants; warps 1-3: the FP64 first element
constexpr int kFirstThreads = 96;

// Row and column of entry e of a packed lower triangle (row-major: (0,0),
// (1,0), (1,1), (2,0), ...).
KS_DEV void tri_rc(int e, int& a, int& b) {
    a = 0;
    while ((a + 1) * (a + 2) / 2 <= e) ++a;
    b = e - a * (a + 1) / 2;
}

// Barrier of the three warps that build the first element (named barrier 1).
KS_DEV void first_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kFirstThreads) : "memory"); }

// The k = 1 element in FP64, by warps 1-3 (thread i of kFirstThreads):
//   m- = F m0 + u, P- = F P0 F^T + Q, v = y - H m- - d, S1 = H P- H^T + R,
//   b1 = m- + (H P-)^T S1^{-1} v,  C1 = P- - (H P-)^T S1^{-1} (H P-).
// GB300 issues one FP64 warp instruction per several tens of cycles on each
// SM sub-partition, so the work is spread over three warps (three
// sub-partitions) and the chain is kept short: the inputs are widened once,
// every stage spreads its entries over the threads (a dot product of length
// N or M each), and S1^{-1} is, for ny <= 3, its adjugate over its
// determinant (leading minors checked), else Gauss-Jordan elimination without
// pivoting by one warp, lane c holding column c of [S1 | I] (S1 is symmetric
// positive definite exactly when every pivot is positive).  p.ok1 = 0 when S1
// is not positive definite.
template <int N, int M, class PS, class MC>
KS_DEV void first_element_fp64(PS& p, MC& mc, int i) {
    constexpr int n1 = kFirstThreads;
    for (int e = i; e < N * N; e += n1) {
        const int a = e / N, b = e % N;
        p.dF[a][b] = (double)p.F[a][b];
        p.dQ[a][b] = 0.5 * ((double)p.Q[a][b] + (double)p.Q[b][a]);
    }
    for (int e = i; e < M * N; e += n1) p.dH[e / N][e % N] = (double)p.H[e / N][e % N];
    for (int e = i; e < M * M; e += n1) {
        const int q = e / M, r = e % M;
        p.dR[q][r] = 0.5 * ((double)p.R[q][r] + (double)p.R[r][q]);
    }
    for (int e = i; e < N; e += n1) p.du[e] = (double)p.u[e];
    for (int e = i; e < M; e += n1) p.v[e] = (double)p.y[e] - (double)p.d[e];
    first_sync();
    for (int e = i; e < N * N + N; e += n1) {          // F P0 and m- = F m0 + u
        if (e < N * N) {
            const int a = e / N, b = e % N;
            double s = 0.0;
            for (int c = 0; c < N; ++c) s = fma(p.dF[a][c], p.P0[c][b], s);
            p.FP[a][b] = s;
        } else {
            const int a = e - N * N;
            double s = p.du[a];
            for (int c = 0; c < N; ++c) s = fma(p.dF[a][c], p.m0[c], s);
            p.mm[a] = s;
        }
    }
    first_sync();
    for (int e = i; e < sym_size(N); e += n1) {        // P- (lower triangle, mirrored)
        int a, b;
        tri_rc(e, a, b);
        double s = p.dQ[a][b];
        for (int c = 0; c < N; ++c) s = fma(p.FP[a][c], p.dF[b][c], s);
        p.Pm[a][b] = s;
        p.Pm[b][a] = s;
    }
    first_sync();
    for (int e = i; e < M * N + M; e += n1) {          // H P- and v = y - d - H m-
        if (e < M * N) {
            const int q = e / N, a = e % N;
            double s = 0.0;
            for (int c = 0; c < N; ++c) s = fma(p.dH[q][c], p.Pm[c][a], s);
            p.HP[q][a] = s;
        } else {
            const int q = e - M * N;
            double s = p.v[q];
            for (int c = 0; c < N; ++c) s = fma(-p.dH[q][c], p.mm[c], s);
            p.v[q] = s;
        }
    }
    first_sync();
    for (int e = i; e < M * M; e += n1) {              // S1 = H P- H^T + R
        const int q = e / M, r = e % M;
        double s = p.dR[q][r];
        for (int c = 0; c < N; ++c) s = fma(p.HP[q][c], p.dH[r][c], s);
        p.S1[q][r] = s;
    }
    first_sync();
    if constexpr (M <= 3) {   // S1^{-1} = adj(S1) / det(S1); thread q * M + r forms the cofactor of (r, q)
        const auto& S = p.S1;
        double cof = 0.0;
        if (i < M * M) {
            const int q = i / M, r = i % M;
            if constexpr (M == 1) {
                cof = 1.0;
            } else if constexpr (M == 2) {
                cof = (q == r) ? S[1 - q][1 - q] : -S[q][r];
            } else {   // 3 x 3: cyclic minors carry their sign
                const int r1 = (r + 1) % 3, r2 = (r + 2) % 3, q1 = (q + 1) % 3, q2 = (q + 2) % 3;
                cof = fma(S[r1][q1], S[r2][q2], -S[r1][q2] * S[r2][q1]);
            }
            p.Si[q][r] = cof;
        }
        first_sync();
        double det = 0.0;   // expansion along row 0: sum_r S[0][r] cof(0, r), cof(0, r) = adj[r][0]
        for (int r = 0; r < M; ++r) det = fma(S[0][r], p.Si[r][0], det);
        bool pd = S[0][0] > 0.0 && det > 0.0;
        if constexpr (M == 3) pd = pd && p.Si[2][2] > 0.0;   // the leading 2 x 2 minor
        const double id = 1.0 / (pd ? det : 1.0);
        first_sync();
        if (i < M * M) p.Si[i / M][i % M] = cof * id;
        if (i == 0 && !pd) p.ok1 = 0;
    } else if (i < 32) {   // Gauss-Jordan on [S1 | I] by the first of the three warps
        static_assert(M <= 16, "one lane per column of [S1 | I]");
        const int c = i;
        double col[M];
#pragma unroll
        for (int r = 0; r < M; ++r) col[r] = c < M ? p.S1[r][c] : (c < 2 * M && r == c - M ? 1.0 : 0.0);
        bool pd = true;
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const double piv = __shfl_sync(0xffffffffu, col[k], k);
            pd = pd && piv > 0.0;
            const double rk = col[k] * (1.0 / (piv > 0.0 ? piv : 1.0));
#pragma unroll
            for (int r = 0; r < M; ++r) {
                if (r == k) continue;
                const double f = __shfl_sync(0xffffffffu, col[r], k);
                col[r] = fma(-f, rk, col[r]);
            }
            col[k] = rk;
        }
        if (c >= M && c < 2 * M) {
#pragma unroll
            for (int r = 0; r < M; ++r) p.Si[r][c - M] = col[r];
        }
        if (c == 0 && !pd) p.ok1 = 0;
    }
    first_sync();
    for (int e = i; e < M * N + M; e += n1) {          // W = S1^{-1} H P-, z = S1^{-1} v
        if (e < M * N) {
            const int q = e / N, a = e % N;
            double s = 0.0;
            for (int r = 0; r < M; ++r) s = fma(p.Si[q][r], p.HP[r][a], s);
            p.W[q][a] = s;
        } else {
            const int q = e - M * N;
            double s = 0.0;
            for (int r = 0; r < M; ++r) s = fma(p.Si[q][r], p.v[r], s);
            p.z[q] = s;
        }
    }
    first_sync();
    for (int e = i; e < sym_size(N) + N; e += n1) {    // C1 = P- - (H P-)^T W, b1 = m- + (H P-)^T z
        if (e < sym_size(N)) {
            int a, b;
            tri_rc(e, a, b);
            double s = p.Pm[a][b];
            for (int q = 0; q < M; ++q) s = fma(-p.HP[q][a], p.W[q][b], s);
            mc.C1[sidx(a, b)] = (float)s;
        } else {
            const int a = e - sym_size(N);
            double s = p.mm[a];
            for (int q = 0; q < M; ++q) s = fma(p.HP[q][a], p.z[q], s);
            mc.b1[a] = (float)s;
        }
    }
}

// One block per model (segment).  After one round of loads, warp 0 builds the
// FP32 constants of Lemma 3 for k > 1 (and the block-fold coefficients), and
// warps 1-3, at the same time, the k = 1 element (prediction of N(m0, P0) and
// update with y_1) in FP64; the two chains only meet for the final store.
// Body of the preparation of segment sg of nseg (one thread block); dyn:
// its dynamic shared memory (PrepSmem and a ModelConst).
// FOLD = false leaves the block-fold coefficient code out (fewer registers
// for launches that never fold).
template <int N, int M, bool FOLD = true>
KS_DEV void prep_body(char* prep_dsm, int sg, int nseg, const float* __restrict__ F, const float* __restrict__ u,
                      const float* __restrict__ Q, const float* __restrict__ H, const float* __restrict__ d,
                      const float* __restrict__ R, const double* __restrict__ m0, const double* __restrict__ P0,
                      const float* __restrict__ y, ModelConst<N, M>* __restrict__ out, uint32_t* __restrict__ status,
                      uint32_t* __restrict__ zero, int nzero, const int64_t* __restrict__ off, int64_t T,
                      const uint32_t* __restrict__ first_tile, BlockCoef<N, M>* __restrict__ coef = nullptr,
                      int ch = 0) {
    PrepSmem<N, M>& p = *reinterpret_cast<PrepSmem<N, M>*>(prep_dsm);
    ModelConst<N, M>& mc =
        *reinterpret_cast<ModelConst<N, M>*>(prep_dsm + ((sizeof(PrepSmem<N, M>) + 15) / 16) * 16);
    const int t = threadIdx.x, nt = blockDim.x;
    const int warp = t >> 5, l = t & 31;
    if (sg == 0) {   // zero[0] is the forward tile counter of the nx <= 6 scans (first_tile: its start)
        for (int i = t; i < nzero; i += nt) zero[i] = (i == 0 && first_tile != nullptr) ? *first_tile : 0u;
        if (t == 0) status[HDR_NEED] = 0u;
    }
    if (off != nullptr && t == 0) {
        const int64_t a = off[sg], b = off[sg + 1];
        const bool okseg = (a < b) && (sg != 0 || a == 0) && (sg != nseg - 1 || b == T);
        if (!okseg) atomicOr(status, ST_BADARG);
    }
    F += (size_t)sg * N * N;
    Q += (size_t)sg * N * N;
    H += (size_t)sg * M * N;
    R += (size_t)sg * M * M;
    m0 += (size_t)sg * N;
    P0 += (size_t)sg * N * N;
    if (u) u += (size_t)sg * N;
    if (d) d += (size_t)sg * M;
    if (y && off) {   // an empty or out-of-range segment has no first measurement
        const int64_t a = off[sg], b = off[sg + 1];
        y = (a >= 0 && a < b && a < T) ? y + a * M : nullptr;
    }
    out += sg;
    // ---- every input in one round of independent loads
    constexpr int nF = N * N, nQ = N * N, nP = N * N, nH = M * N, nR = M * M;
    constexpr int nAll = nF + nQ + nP + nH + nR + N + N + M + M;
    for (int e = t; e < nAll; e += nt) {
        int i = e;
        if (i < nF) { p.F[i / N][i % N] = F[i]; continue; }
        i -= nF;
        if (i < nQ) { p.Q[i / N][i % N] = Q[i]; continue; }
        i -= nQ;
        if (i < nP) { p.P0[i / N][i % N] = P0[i]; continue; }
        i -= nP;
        if (i < nH) { p.H[i / N][i % N] = H[i]; continue; }
        i -= nH;
        if (i < nR) { p.R[i / M][i % M] = R[i]; continue; }
        i -= nR;
        if (i < N) { p.u[i] = u ? u[i] : 0.f; continue; }
        i -= N;
        if (i < N) { p.m0[i] = m0[i]; continue; }
        i -= N;
        if (i < M) { p.d[i] = d ? d[i] : 0.f; continue; }
        i -= M;
        p.y[i] = y ? y[i] : 0.f;
    }
    if (t == 0) { p.ok0 = 1; p.ok1 = 1; }
    __syncthreads();

    if (warp == 0) {
        // ---- FP32 constants for k > 1: S = H Q H^T + R = L_S L_S^T, U = L_S^{-1} H F,
        // K = Q H^T S^{-1}, A = F - K H F, C = Q - K S K^T (Q, R symmetrised)
        for (int e = l; e < M * N; e += 32) {
            const int q = e / N, a = e % N;
            float s = 0.f, h = 0.f;
            for (int c = 0; c < N; ++c) {
                s = fmaf(p.H[q][c], 0.5f * (p.Q[c][a] + p.Q[a][c]), s);
                h = fmaf(p.H[q][c], p.F[c][a], h);
            }
            p.HQ[q][a] = s;
            p.HF[q][a] = h;
        }
        __syncwarp();
        for (int e = l; e < M * M; e += 32) {
            const int q = e / M, r = e % M;
            float s = 0.5f * (p.R[q][r] + p.R[r][q]);
            for (int c = 0; c < N; ++c) s = fmaf(p.HQ[q][c], p.H[r][c], s);
            p.S[q][r] = s;
        }
        __syncwarp();
        if (l == 0) {                              // Cholesky of S, L_S^{-1}
            float Ls[M][M];
            bool ok = true;
            for (int j = 0; j < M; ++j) {
                float s = p.S[j][j];
                for (int k = 0; k < j; ++k) s -= Ls[j][k] * Ls[j][k];
                ok = ok && (s > 0.f);
                Ls[j][j] = sqrtf(fmaxf(s, 1e-37f));
                for (int i = j + 1; i < M; ++i) {
                    float q = p.S[i][j];
                    for (int k = 0; k < j; ++k) q -= Ls[i][k] * Ls[j][k];
                    Ls[i][j] = q / Ls[j][j];
                }
            }
            for (int c = 0; c < M; ++c)
                for (int i = 0; i < M; ++i) {
                    if (i < c) { p.Lsi[i][c] = 0.f; continue; }
                    float q = (i == c) ? 1.f : 0.f;
                    for (int k = c; k < i; ++k) q -= Ls[i][k] * p.Lsi[k][c];
                    p.Lsi[i][c] = q / Ls[i][i];
                }
            if (!ok) p.ok0 = 0;
        }
        __syncwarp();
        for (int e = l; e < M * N; e += 32) {      // tmp = L_S^{-1} H Q, U = L_S^{-1} H F
            const int q = e / N, a = e % N;
            float s = 0.f, v = 0.f;
            for (int r = 0; r <= q; ++r) { s = fmaf(p.Lsi[q][r], p.HQ[r][a], s); v = fmaf(p.Lsi[q][r], p.HF[r][a], v); }
            p.tmp[q][a] = s;
            mc.U[q * N + a] = v;
        }
        for (int e = l; e < M; e += 32) {
            float s = p.d[e];
            for (int c = 0; c < N; ++c) s = fmaf(p.H[e][c], p.u[c], s);
            mc.hud[e] = s;
            for (int r = 0; r < M; ++r) mc.Lsi[e * M + r] = p.Lsi[e][r];
        }
        __syncwarp();
        for (int e = l; e < N * M; e += 32) {      // K = tmp^T L_S^{-1}
            const int a = e / M, q = e % M;
            float s = 0.f;
            for (int r = q; r < M; ++r) s = fmaf(p.tmp[r][a], p.Lsi[r][q], s);
            p.K[a][q] = s;
            mc.K[a * M + q] = s;
        }
        __syncwarp();
        for (int e = l; e < N * N; e += 32) {      // A = F - K H F ; C = Q - tmp^T tmp ; copies
            const int a = e / N, b = e % N;
            float s = p.F[a][b];
            for (int q = 0; q < M; ++q) s = fmaf(-p.K[a][q], p.HF[q][b], s);
            mc.A[a * N + b] = s;
            mc.F[a * N + b] = p.F[a][b];
            if (b <= a) {
                const float qs = 0.5f * (p.Q[a][b] + p.Q[b][a]);
                float c = qs;
                for (int q = 0; q < M; ++q) c = fmaf(-p.tmp[q][a], p.tmp[q][b], c);
                mc.C[sidx(a, b)] = c;
                mc.Q[sidx(a, b)] = qs;
            }
        }
        for (int e = l; e < N; e += 32) mc.u[e] = p.u[e];
        if (l < 4) mc.pad[l] = 0.f;
        if constexpr (N <= 6 && FOLD) {   // register-path sizes only
            if (coef != nullptr) {   // the block-fold coefficients, while warps 1-3 build the k = 1 element
                __syncwarp();
                block_coef_warp<N, M>(mc, &p.H[0][0], ch, coef + sg);
            }
        }
    } else {   // warps 1-3
        if (y != nullptr) {
            first_element_fp64<N, M>(p, mc, t - 32);
        } else {
            for (int e = t - 32; e < N; e += kFirstThreads) mc.b1[e] = 0.f;
            for (int e = t - 32; e < sym_size(N); e += kFirstThreads) mc.C1[e] = 0.f;
        }
    }
    __syncthreads();
    {
        const float* src = reinterpret_cast<const float*>(&mc);
        float* dst = reinterpret_cast<float*>(out);
        for (int i = t; i < (int)(sizeof(ModelConst<N, M>) / 4); i += nt) dst[i] = src[i];
    }
    if (t == 0 && !(p.ok0 && p.ok1)) atomicOr(status, ST_NUMERIC);
}

// Dynamic shared memory of prep_body.
template <int N, int M>
constexpr size_t prep_dyn_smem() {
    return ((sizeof(PrepSmem<N, M>) + 15) / 16) * 16 + sizeof(ModelConst<N, M>) + 16;
}

// One block per model (segment); block 0 also zeroes the scans' counters and
// flags (`zero`), the first one from *first_tile when given.
template <int N, int M, bool FOLD = true>
__global__ void __launch_bounds__(kPrepThreads) prep_kernel(const float* __restrict__ F, const float* __restrict__ u,
                                                   const float* __restrict__ Q, const float* __restrict__ H,
                                                   const float* __restrict__ d, const float* __restrict__ R,
                                                   const double* __restrict__ m0, const double* __restrict__ P0,
                                                   const float* __restrict__ y, ModelConst<N, M>* __restrict__ out,
                                                   uint32_t* __restrict__ status, uint32_t* __restrict__ zero,
                                                   int nzero, const int64_t* __restrict__ off, int64_t T,
                                                   const uint32_t* __restrict__ first_tile = nullptr,
                                                   BlockCoef<N, M>* __restrict__ coef = nullptr, int ch = 0) {
    extern __shared__ __align__(16) char prep_dsm[];
    pdl_wait();
    prep_body<N, M, FOLD>(prep_dsm, (int)blockIdx.x, (int)gridDim.x, F, u, Q, H, d, R, m0, P0, y, out, status, zero,
                          nzero, off, T, first_tile, coef, ch);
    pdl_trigger();
}

// ---------------------------------------------------------------- Lemma 3 materialised
// Element k written component-major: component c of element k at el[c*ld + k],
// A [N*N], b [N], C [N*N], eta [N], J [N*N] (full, symmetric).
template <int N, int M>
__global__ void __launch_bounds__(256) build_elements_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                             const float* __restrict__ y, int64_t T,
                                                             float* __restrict__ el, int64_t ld) {
    __shared__ ModelConst<N, M> mc;
    load_const<N, M>(mcg, mc, threadIdx.x, blockDim.x);
    __syncthreads();
    constexpr int ob = N * N, oC = N * N + N, oe = 2 * N * N + N, oJ = 2 * N * N + 2 * N;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < T;
         k += (int64_t)gridDim.x * blockDim.x) {
        FElem<N> e;
        if (k == 0) {
            first_element<N, M>(mc, e);
        } else {
            float yk[M], b[N], w[M];
            load_meas<M>(y, k, yk);
            meas_element<N, M>(mc, yk, b, w);
            expand_meas<N, M>(mc, b, w, e);
        }
#pragma unroll
        for (int a = 0; a < N * N; ++a) el[a * ld + k] = e.A[a];
#pragma unroll
        for (int a = 0; a < N; ++a) {
            el[(ob + a) * ld + k] = e.b[a];
            el[(oe + a) * ld + k] = e.eta[a];
        }
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b < N; ++b) {
                el[(oC + a * N + b) * ld + k] = e.C[sidx(a, b)];
                el[(oJ + a * N + b) * ld + k] = e.J[sidx(a, b)];
            }
    }
}

// ---------------------------------------------------------------- Lemma 3, time-varying
// Filtering element of a time-varying model in its measurement form: A, b,
// C and (U, w) with eta = U^T w and J = U^T U (rank ny), so that the scans
// combine it with the rank-ny operators of a time-invariant model.  Stored
// per step as one contiguous record of kFloats (a multiple of 4).
template <int N, int M>
struct TVElem {
    static constexpr int kFloats = N * N + sym_size(N) + M * N + N + M;
    static_assert(kFloats % 4 == 0, "records are moved as float4");
    float A[N * N];
    float C[sym_size(N)];
    float U[M * N];
    float b[N];
    float w[M];
};

template <int N, int M>
KS_DEV void store_tvelem(float* __restrict__ el, int64_t k, const TVElem<N, M>& e) {
    static_assert(sizeof(TVElem<N, M>) == 4 * TVElem<N, M>::kFloats, "packed record");
    const float4* src = reinterpret_cast<const float4*>(&e);
    float4* dst = reinterpret_cast<float4*>(el + k * TVElem<N, M>::kFloats);
#pragma unroll
    for (int i = 0; i < TVElem<N, M>::kFloats / 4; ++i) dst[i] = src[i];
}

template <int N, int M>
KS_DEV void load_tvelem(const float* __restrict__ el, int64_t k, TVElem<N, M>& e) {
    const float4* src = reinterpret_cast<const float4*>(el + k * TVElem<N, M>::kFloats);
    float4* dst = reinterpret_cast<float4*>(&e);
#pragma unroll
    for (int i = 0; i < TVElem<N, M>::kFloats / 4; ++i) dst[i] = __ldg(src + i);
}

// Step k >= 1 from that step's (F, u, Q) and (H, d, R).  With
// S = H Q H^T + R = L L^T (Cholesky), U = L^{-1} H F, V = L^{-1} H Q and
// w = L^{-1} (y - H u - d), Lemma 3's gain is K = Q H^T S^{-1} = V^T L^{-1}, so
//   A = F - V^T U,  b = u + V^T w,  C = Q - V^T V,  eta = U^T w,  J = U^T U.
template <int N, int M>
KS_DEV void tv_element(const TVArgs& tv, const float* __restrict__ y, int64_t k, TVElem<N, M>& e, Flags& bad) {
    float F[N][N], Q[N][N], H[M][N], R[M][M], u[N], d[M], yk[M];
    {
        float Qr[N * N], Rr[M * M];
        load_step<N * N>(tv.F, k, &F[0][0]);
        load_step<N * N>(tv.Q, k, Qr);
        load_step<M * N>(tv.H, k, &H[0][0]);
        load_step<M * M>(tv.R, k, Rr);
        load_step<M>(y, k, yk);
        if (tv.u) load_step<N>(tv.u, k, u);
        else {
#pragma unroll
            for (int a = 0; a < N; ++a) u[a] = 0.f;
        }
        if (tv.d) load_step<M>(tv.d, k, d);
        else {
#pragma unroll
            for (int q = 0; q < M; ++q) d[q] = 0.f;
        }
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) Q[a][b] = Q[b][a] = 0.5f * (Qr[a * N + b] + Qr[b * N + a]);
#pragma unroll
        for (int q = 0; q < M; ++q)
#pragma unroll
            for (int r = 0; r <= q; ++r) R[q][r] = 0.5f * (Rr[q * M + r] + Rr[r * M + q]);
    }
    float HF[M][N], HQ[M][N], r0[M];
#pragma unroll
    for (int q = 0; q < M; ++q) {
        float hu = d[q];
#pragma unroll
        for (int a = 0; a < N; ++a) {
            float f = 0.f, g = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) { f = fmaf(H[q][c], F[c][a], f); g = fmaf(H[q][c], Q[c][a], g); }
            HF[q][a] = f;
            HQ[q][a] = g;
            hu = fmaf(H[q][a], u[a], hu);
        }
        r0[q] = yk[q] - hu;
    }
    float L[M][M], rd[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        float s = R[j][j];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(HQ[j][c], H[j][c], s);
#pragma unroll
        for (int l = 0; l < j; ++l) s = fmaf(-L[j][l], L[j][l], s);
        bad |= !(s > 0.f);
        const float r = rsqrtf(fmaxf(s, 1e-37f));
        L[j][j] = s * r;
        rd[j] = r;
#pragma unroll
        for (int i = j + 1; i < M; ++i) {
            float t = R[i][j];
#pragma unroll
            for (int c = 0; c < N; ++c) t = fmaf(HQ[i][c], H[j][c], t);
#pragma unroll
            for (int l = 0; l < j; ++l) t = fmaf(-L[i][l], L[j][l], t);
            L[i][j] = t * r;
        }
    }
    float V[M][N];   // forward substitution with L
#pragma unroll
    for (int i = 0; i < M; ++i) {
        float t = r0[i];
#pragma unroll
        for (int l = 0; l < i; ++l) t = fmaf(-L[i][l], e.w[l], t);
        e.w[i] = t * rd[i];
#pragma unroll
        for (int a = 0; a < N; ++a) {
            float x = HF[i][a], v = HQ[i][a];
#pragma unroll
            for (int l = 0; l < i; ++l) { x = fmaf(-L[i][l], e.U[l * N + a], x); v = fmaf(-L[i][l], V[l][a], v); }
            e.U[i * N + a] = x * rd[i];
            V[i][a] = v * rd[i];
        }
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float bb = u[a];
#pragma unroll
        for (int q = 0; q < M; ++q) bb = fmaf(V[q][a], e.w[q], bb);
        e.b[a] = bb;
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float x = F[a][b];
#pragma unroll
            for (int q = 0; q < M; ++q) x = fmaf(-V[q][a], e.U[q * N + b], x);
            e.A[a * N + b] = x;
        }
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            float c = Q[a][b];
#pragma unroll
            for (int q = 0; q < M; ++q) c = fmaf(-V[q][a], V[q][b], c);
            e.C[sidx(a, b)] = c;
        }
    }
}

// Step 0 of a time-varying model (Lemma 3, k = 1) in FP64: the prior N(m0, P0)
// is predicted with (F[0], u[0], Q[0]) and updated with y[0]; A = 0 and
// U = w = 0, i.e. eta = J = 0 (the element does not depend on the state
// before it).
template <int N, int M>
__device__ __noinline__ void tv_first_element(const TVArgs& tv, const float* __restrict__ y, TVElem<N, M>& e,
                                              Flags& bad) {
    double Pm[N][N], mm[N], HP[M][N], S[M][M], L[M][M], t1[M][N], z[M];
    for (int a = 0; a < N; ++a) {
        double s = tv.u ? (double)tv.u[a] : 0.0;
        for (int c = 0; c < N; ++c) s += (double)tv.F[a * N + c] * tv.m0[c];
        mm[a] = s;
    }
    for (int a = 0; a < N; ++a)
        for (int b = 0; b <= a; ++b) {           // P- = F P0 F^T + Q (lower, mirrored)
            double s = 0.5 * ((double)tv.Q[a * N + b] + (double)tv.Q[b * N + a]);
            for (int c = 0; c < N; ++c) {
                double fp = 0.0;                 // (F P0)[a][c]
                for (int l = 0; l < N; ++l) fp += (double)tv.F[a * N + l] * tv.P0[l * N + c];
                s += fp * (double)tv.F[b * N + c];
            }
            Pm[a][b] = Pm[b][a] = s;
        }
    for (int q = 0; q < M; ++q)
        for (int a = 0; a < N; ++a) {
            double s = 0.0;
            for (int c = 0; c < N; ++c) s += (double)tv.H[q * N + c] * Pm[c][a];
            HP[q][a] = s;
        }
    for (int q = 0; q < M; ++q)
        for (int r = 0; r <= q; ++r) {
            double s = 0.5 * ((double)tv.R[q * M + r] + (double)tv.R[r * M + q]);
            for (int c = 0; c < N; ++c) s += HP[q][c] * (double)tv.H[r * N + c];
            S[q][r] = s;
        }
    for (int j = 0; j < M; ++j) {               // Cholesky S = L L^T
        double s = S[j][j];
        for (int l = 0; l < j; ++l) s -= L[j][l] * L[j][l];
        bad |= !(s > 0.0);
        L[j][j] = sqrt(s > 0.0 ? s : 1e-300);
        for (int i = j + 1; i < M; ++i) {
            double t = S[i][j];
            for (int l = 0; l < j; ++l) t -= L[i][l] * L[j][l];
            L[i][j] = t / L[j][j];
        }
    }
    for (int q = 0; q < M; ++q) {               // z = L^{-1} (y - H m- - d), t1 = L^{-1} H P-
        double s = (double)y[q] - (tv.d ? (double)tv.d[q] : 0.0);
        for (int c = 0; c < N; ++c) s -= (double)tv.H[q * N + c] * mm[c];
        for (int l = 0; l < q; ++l) s -= L[q][l] * z[l];
        z[q] = s / L[q][q];
        for (int a = 0; a < N; ++a) {
            double t = HP[q][a];
            for (int l = 0; l < q; ++l) t -= L[q][l] * t1[l][a];
            t1[q][a] = t / L[q][q];
        }
    }
    for (int a = 0; a < N; ++a) {               // b = m- + t1^T z, C = P- - t1^T t1
        double s = mm[a];
        for (int q = 0; q < M; ++q) s += t1[q][a] * z[q];
        e.b[a] = (float)s;
        for (int b = 0; b < N; ++b) e.A[a * N + b] = 0.f;
        for (int b = 0; b <= a; ++b) {
            double c = Pm[a][b];
            for (int q = 0; q < M; ++q) c -= t1[q][a] * t1[q][b];
            e.C[sidx(a, b)] = (float)c;
        }
    }
    for (int a = 0; a < M * N; ++a) e.U[a] = 0.f;
    for (int q = 0; q < M; ++q) e.w[q] = 0.f;
}

// Filtering elements of a time-varying model, one TVElem record per step
// (el must be 16-byte aligned).  Block 0 also clears the scans' counters and
// flags.
template <int N, int M>
__global__ void __launch_bounds__(256) tv_elements_kernel(TVArgs tv, const float* __restrict__ y, int64_t T,
                                                          float* __restrict__ el, uint32_t* __restrict__ status,
                                                          uint32_t* __restrict__ zero, int nzero) {
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < nzero; i += blockDim.x) zero[i] = 0u;
        if (threadIdx.x == 0) status[HDR_NEED] = 0u;
    }
    Flags bad = 0u;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < T;
         k += (int64_t)gridDim.x * blockDim.x) {
        TVElem<N, M> e;
        if (k == 0) tv_first_element<N, M>(tv, y, e, bad);
        else tv_element<N, M>(tv, y, k, e, bad);
        store_tvelem<N, M>(el, k, e);
    }
    report_flags(status, bad, kFull, (threadIdx.x & 31) == 0);
}

// Per-step model constants of a time-varying model (steps 1..T-1; step 0,
// with its k = 1 element, comes from prep_kernel): the FP32 part of
// prep_kernel evaluated per step by one thread, for the kernels that read
// their model through a Cursor (one warp per chain).
template <int N, int M>
__global__ void __launch_bounds__(128) tv_const_kernel(TVArgs tv, int64_t T, ModelConst<N, M>* __restrict__ out,
                                                       uint32_t* __restrict__ status) {
    Flags bad = 0u;
    for (int64_t k = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < T;
         k += (int64_t)gridDim.x * blockDim.x) {
        ModelConst<N, M>& mc = out[k];
        float F[N * N], Q[N * N], H[M * N], R[M * M], u[N], d[M];
        load_step<N * N>(tv.F, k, F);
        load_step<N * N>(tv.Q, k, Q);
        load_step<M * N>(tv.H, k, H);
        load_step<M * M>(tv.R, k, R);
        if (tv.u) load_step<N>(tv.u, k, u);
        else {
#pragma unroll
            for (int a = 0; a < N; ++a) u[a] = 0.f;
        }
        if (tv.d) load_step<M>(tv.d, k, d);
        else {
#pragma unroll
            for (int q = 0; q < M; ++q) d[q] = 0.f;
        }
        float HQ[M][N], HF[M][N];
        for (int q = 0; q < M; ++q)
            for (int a = 0; a < N; ++a) {
                float sq = 0.f, sf = 0.f;
                for (int c = 0; c < N; ++c) {
                    sq = fmaf(H[q * N + c], 0.5f * (Q[c * N + a] + Q[a * N + c]), sq);
                    sf = fmaf(H[q * N + c], F[c * N + a], sf);
                }
                HQ[q][a] = sq;
                HF[q][a] = sf;
            }
        float Ls[M][M], Lsi[M][M];
        for (int j = 0; j < M; ++j) {
            float sj = 0.5f * (R[j * M + j] + R[j * M + j]);
            for (int c = 0; c < N; ++c) sj = fmaf(HQ[j][c], H[j * N + c], sj);
            for (int l = 0; l < j; ++l) sj = fmaf(-Ls[j][l], Ls[j][l], sj);
            bad |= !(sj > 0.f);
            const float rj = rsqrtf(fmaxf(sj, 1e-37f));
            Ls[j][j] = sj * rj;
            for (int i = j + 1; i < M; ++i) {
                float t = 0.5f * (R[i * M + j] + R[j * M + i]);
                for (int c = 0; c < N; ++c) t = fmaf(HQ[i][c], H[j * N + c], t);
                for (int l = 0; l < j; ++l) t = fmaf(-Ls[i][l], Ls[j][l], t);
                Ls[i][j] = t * rj;
            }
        }
        for (int c = 0; c < M; ++c)                // L_S^{-1}, column by column
            for (int i = 0; i < M; ++i) {
                if (i < c) { Lsi[i][c] = 0.f; continue; }
                float t = (i == c) ? 1.f : 0.f;
                for (int l = c; l < i; ++l) t = fmaf(-Ls[i][l], Lsi[l][c], t);
                Lsi[i][c] = t / Ls[i][i];
            }
        float tmp[M][N];
        for (int q = 0; q < M; ++q)
            for (int a = 0; a < N; ++a) {
                float st = 0.f, sv = 0.f;
                for (int r = 0; r <= q; ++r) { st = fmaf(Lsi[q][r], HQ[r][a], st); sv = fmaf(Lsi[q][r], HF[r][a], sv); }
                tmp[q][a] = st;
                mc.U[q * N + a] = sv;
            }
        for (int q = 0; q < M; ++q) {
            float hu = d[q];
            for (int c = 0; c < N; ++c) hu = fmaf(H[q * N + c], u[c], hu);
            mc.hud[q] = hu;
            for (int r = 0; r < M; ++r) mc.Lsi[q * M + r] = Lsi[q][r];
        }
        for (int a = 0; a < N; ++a)
            for (int q = 0; q < M; ++q) {
                float sk = 0.f;
                for (int r = q; r < M; ++r) sk = fmaf(tmp[r][a], Lsi[r][q], sk);
                mc.K[a * M + q] = sk;
            }
        for (int a = 0; a < N; ++a) {
            for (int b = 0; b < N; ++b) {
                float sa = F[a * N + b];
                for (int q = 0; q < M; ++q) sa = fmaf(-mc.K[a * M + q], HF[q][b], sa);
                mc.A[a * N + b] = sa;
                mc.F[a * N + b] = F[a * N + b];
            }
            for (int b = 0; b <= a; ++b) {
                const float qs = 0.5f * (Q[a * N + b] + Q[b * N + a]);
                float c = qs;
                for (int q = 0; q < M; ++q) c = fmaf(-tmp[q][a], tmp[q][b], c);
                mc.C[sidx(a, b)] = c;
                mc.Q[sidx(a, b)] = qs;
            }
            mc.u[a] = u[a];
            mc.b1[a] = 0.f;
        }
        for (int a = 0; a < sym_size(N); ++a) mc.C1[a] = 0.f;
        for (int a = 0; a < 4; ++a) mc.pad[a] = 0.f;
    }
    report_flags(status, bad, kFull, (threadIdx.x & 31) == 0);
}

// ---------------------------------------------------------------- staging
// Outputs (and, for the reverse scan, inputs) of each thread's block of steps
// are staged in shared memory in groups of G steps and moved with per-thread
// bulk copies (TMA), so that global traffic is contiguous 16-byte-aligned
// runs instead of one scattered row per step.  Used when a mean row (4 nx
// bytes) is a multiple of 16 bytes; otherwise rows go straight to memory.
template <int N>
struct Stage {
    static constexpr bool kOn = (N % 4) == 0;
    static constexpr int G = 4;                                   // steps per group
    static constexpr int kMeanB = 4 * N, kCovB = 4 * N * N;       // bytes per step
    static constexpr int kBuf = G * (kMeanB + kCovB);             // one group
    // per-thread stride: an odd number of 16-byte units keeps the 8 threads of
    // a quarter warp on distinct banks for 16-byte accesses
    __host__ __device__ static constexpr int pad_odd(int b) { return ((b / 16) % 2 == 1) ? b : b + 16; }
};

template <int N>
KS_DEV void stage_write(char* buf, int slot, const float (&m)[N], const float (&S)[sym_size(N)]) {
    constexpr int G = Stage<N>::G;
    float* pm = reinterpret_cast<float*>(buf) + slot * N;
    float* pc = reinterpret_cast<float*>(buf + G * Stage<N>::kMeanB) + slot * N * N;
#pragma unroll
    for (int i = 0; i < N; i += 4) *reinterpret_cast<float4*>(pm + i) = make_float4(m[i], m[i + 1], m[i + 2], m[i + 3]);
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int i = 0; i < N; i += 4)
            *reinterpret_cast<float4*>(pc + a * N + i) =
                make_float4(S[sidx(a, i)], S[sidx(a, i + 1)], S[sidx(a, i + 2)], S[sidx(a, i + 3)]);
}

template <int N>
KS_DEV void stage_read(const char* buf, int slot, float (&m)[N], float (&S)[sym_size(N)]) {
    constexpr int G = Stage<N>::G;
    const float* pm = reinterpret_cast<const float*>(buf) + slot * N;
    const float* pc = reinterpret_cast<const float*>(buf + G * Stage<N>::kMeanB) + slot * N * N;
#pragma unroll
    for (int i = 0; i < N; i += 4) {
        const float4 t = *reinterpret_cast<const float4*>(pm + i);
        m[i] = t.x; m[i + 1] = t.y; m[i + 2] = t.z; m[i + 3] = t.w;
    }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int i = 0; i < N; i += 4) {
            const float4 t = *reinterpret_cast<const float4*>(pc + a * N + i);
            if (i <= a) S[sidx(a, i)] = t.x;
            if (i + 1 <= a) S[sidx(a, i + 1)] = t.y;
            if (i + 2 <= a) S[sidx(a, i + 2)] = t.z;
            if (i + 3 <= a) S[sidx(a, i + 3)] = t.w;
        }
}

// Group of `cnt` steps starting at step k0 (mean rows then covariance rows of
// the group in `buf`) to global memory.
template <int N>
KS_DEV void stage_flush(char* buf, float* mean, float* cov, int64_t k0, int cnt) {
    constexpr int G = Stage<N>::G;
    fence_proxy_async();
    bulk_store(mean + k0 * N, buf, (uint32_t)(cnt * Stage<N>::kMeanB));
    bulk_store(cov + k0 * N * N, buf + G * Stage<N>::kMeanB, (uint32_t)(cnt * Stage<N>::kCovB));
    bulk_commit();
}

template <int N>
KS_DEV void stage_fetch(char* buf, const float* mean, const float* cov, int64_t k0, int cnt, uint64_t* mb) {
    constexpr int G = Stage<N>::G;
    fence_proxy_async();
    mbar_expect_tx(mb, (uint32_t)(cnt * (Stage<N>::kMeanB + Stage<N>::kCovB)));
    bulk_load(buf, mean + k0 * N, (uint32_t)(cnt * Stage<N>::kMeanB), mb);
    bulk_load(buf + G * Stage<N>::kMeanB, cov + k0 * N * N, (uint32_t)(cnt * Stage<N>::kCovB), mb);
}

// ---------------------------------------------------------------- look-back
// Decoupled look-back by one warp over windows of 32 predecessor tiles.  Lane
// l inspects tile base - l.  If some tile in the window has published its
// inclusive prefix, the nearest one (lane p) is used and the aggregates of
// the p tiles after it are reduced in log2(p) shuffle levels; otherwise all
// 32 aggregates are reduced and the window moves back.  Returns (in lane 0)
// the exclusive prefix of `tile`, in prefix form.
//   Op::combine(x, y)   x (x) y for general elements, x earlier in scan order
//   Op::advance(st, e)  prefix-form state (x) general element
template <class Op>
KS_DEV typename Op::State lookback_warp(const ScanState& ss, int tile, int lane, Flags& bad, bool& timeout) {
    using E = typename Op::Elem;
    using S = typename Op::State;
    constexpr int AF = sizeof(E) / 4, PF = sizeof(S) / 4;
    S ex;
    E run;
    bool have_run = false;
    int base = tile - 1;
    const uint32_t limit = wait_limit(ss);
    while (true) {
        const int j = base - lane;
        uint32_t f = 0u;
        if (j >= 0) f = wait_flag(ss.flags + j, limit);
        const bool lost = (j >= 0) && (f == 0u);
        if (__any_sync(kFull, lost)) {
            timeout = true;
            Op::zero_state(ex);
            return ex;
        }
        const unsigned pm = __ballot_sync(kFull, (j >= 0) && (f == kFlagPre));
        const int p = pm ? (__ffs(pm) - 1) : 32;
        E x;
        if (lane < p && j >= 0) x = load_cg<E>(ss.agg + (int64_t)j * AF);
        else Op::identity(x);
#pragma unroll 1
        for (int d = 1; d < p; d <<= 1) {
            const E o = shfl_down_t(x, d);      // lane + d holds an earlier tile
            if ((lane & (2 * d - 1)) == 0) x = Op::combine(o, x, bad);
        }
        if (p < 32) {
            if (lane == 0) {
                ex = load_cg<S>(ss.pre + (int64_t)(base - p) * PF);
                if (p > 0) Op::advance(ex, x, bad);
                if (have_run) Op::advance(ex, run, bad);
            }
            return ex;
        }
        if (lane == 0) {
            run = have_run ? Op::combine(x, run, bad) : x;
            have_run = true;
        }
        base -= 32;
    }
}

template <int N, int REF = REF_FP64>
struct FilterOp {
    using Elem = FElem<N>;
    using State = FState<N>;
    KS_DEV static Elem combine(const Elem& a, const Elem& b, Flags& bad) { return fcombine<N, REF>(a, b, bad); }
    KS_DEV static void advance(State& s, const Elem& e, Flags& bad) { fadvance<N, REF>(s, e, bad); }
    KS_DEV static void identity(Elem& e) { set_identity<N>(e); }
    KS_DEV static void zero_state(State& s) {
#pragma unroll
        for (int a = 0; a < N; ++a) s.b[a] = 0.f;
#pragma unroll
        for (int a = 0; a < sym_size(N); ++a) s.C[a] = 0.f;
    }
    KS_DEV static State state_of(const Elem& e) {   // element with A = 0
        State s;
#pragma unroll
        for (int a = 0; a < N; ++a) s.b[a] = e.b[a];
#pragma unroll
        for (int a = 0; a < sym_size(N); ++a) s.C[a] = e.C[a];
        return s;
    }
};

// Reverse-scan operator in scan (reversed-time) order: x (x)_r y = y (x) x.
template <int N>
struct SmootherOp {
    using Elem = SElem<N>;
    using State = SState<N>;
    KS_DEV static Elem combine(const Elem& a, const Elem& b, Flags&) { return scombine<N>(b, a); }
    KS_DEV static void advance(State& s, const Elem& e, Flags&) { sadvance<N>(e, s); }
    KS_DEV static void identity(Elem& e) { set_identity<N>(e); }
    KS_DEV static void zero_state(State& s) {
#pragma unroll
        for (int a = 0; a < N; ++a) s.g[a] = 0.f;
#pragma unroll
        for (int a = 0; a < sym_size(N); ++a) s.L[a] = 0.f;
    }
    KS_DEV static State state_of(const Elem& e) {   // element with E = 0
        State s;
#pragma unroll
        for (int a = 0; a < N; ++a) s.g[a] = e.g[a];
#pragma unroll
        for (int a = 0; a < sym_size(N); ++a) s.L[a] = e.L[a];
        return s;
    }
};

// Phase 2 shared by both scans: warp scan of the per-thread block elements,
// scan of the warp totals (last warp, NW lanes), publication of the tile
// aggregate and the look-back.  On return every thread of a valid block has
// `st` = the prefix entering its block and `has` = whether there is one (only
// the very first block of the sequence has none).
template <class E, class S, int NT>
struct BlockScanSmem {
    E wtot[NT / 32];
    E wincl[NT / 32];
    E lexcl[NT];     // per-thread in-warp exclusive prefix, parked across the look-back
    E tagg;
    S texcl;
    int has;
};

// LOp: the operator of the look-back (the same operator; a variant may differ
// in how it takes its inverses).
template <class Op, int NT, class LOp = Op>
struct BlockScan {
    static constexpr int NW = NT / 32;
    using E = typename Op::Elem;
    using S = typename Op::State;
    using Smem = BlockScanSmem<E, S, NT>;

    KS_DEV static void run(Smem& sm, const ScanState& ss, int tile, const E& acc, S& st, bool& has,
                           Flags& bad) {
        const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
        constexpr int AF = sizeof(E) / 4, PF = sizeof(S) / 4;
        E incl = acc;
#pragma unroll 1
        for (int d = 1; d < 32; d <<= 1) {
            const E o = shfl_up_t(incl, d);
            if (lane >= d) incl = Op::combine(o, incl, bad);
        }
        {
            const E lane_excl = shfl_up_t(incl, 1);
            sm.lexcl[tid] = lane_excl;
        }
        if (lane == 31) sm.wtot[warp] = incl;
        __syncthreads();
        if (warp == NW - 1) {
            {
                E x;
                if (lane < NW) x = sm.wtot[lane];
                else Op::identity(x);
#pragma unroll 1
                for (int d = 1; d < NW; d <<= 1) {
                    const E o = shfl_up_t(x, d);
                    if (lane >= d && lane < NW) x = Op::combine(o, x, bad);
                }
                if (lane < NW) sm.wincl[lane] = x;
                if (lane == NW - 1) sm.tagg = x;
            }
            __syncwarp();
            bool timeout = false;
            S ex;
            if (tile == 0) {
                if (lane == 0) {
                    store_plain(ss.pre, Op::state_of(sm.tagg));
                    st_release(ss.flags, kFlagPre);
                }
            } else {
                if (lane == 0) {
                    store_plain(ss.agg + (int64_t)tile * AF, sm.tagg);
                    st_release(ss.flags + tile, kFlagAgg);
                }
                ex = lookback_warp<LOp>(ss, tile, lane, bad, timeout);
                if (lane == 0) {
                    S inc = ex;
                    LOp::advance(inc, sm.tagg, bad);
                    store_plain(ss.pre + (int64_t)tile * PF, inc);
                    st_release(ss.flags + tile, kFlagPre);
                }
            }
            if (timeout && lane == 0) atomicOr(ss.status, ST_TIMEOUT);
            if (lane == 0) {
                if (tile != 0) sm.texcl = ex;
                sm.has = (tile != 0) ? 1 : 0;
            }
        }
        __syncthreads();
        has = sm.has != 0;
        if (has) st = sm.texcl;
        if (warp > 0) {
            const E& wp = sm.wincl[warp - 1];
            if (has) Op::advance(st, wp, bad);
            else { st = Op::state_of(wp); has = true; }
        }
        if (lane > 0) {
            const E& le = sm.lexcl[tid];
            if (has) Op::advance(st, le, bad);
            else { st = Op::state_of(le); has = true; }
        }
    }
};

// Lemma 5 element from a filtered mean and covariance (k = n when `last`).
template <int N, int M, class MC>
KS_DEV void build_selem_from(const MC& mc, const float (&xb)[N], const float (&P)[sym_size(N)],
                             bool last, SElem<N>& e, Flags& bad) {
    if (last) {  // Lemma 5, k = n: E = 0, g = xbar_n, L = P_n
#pragma unroll
        for (int a = 0; a < N * N; ++a) e.E[a] = 0.f;
#pragma unroll
        for (int a = 0; a < N; ++a) e.g[a] = xb[a];
#pragma unroll
        for (int a = 0; a < sym_size(N); ++a) e.L[a] = P[a];
    } else {
        smoother_element<N, M>(mc, xb, P, e, bad);
    }
}

// ---------------------------------------------------------------- forward scan
// With SAGG the same pass also builds each step's Lemma 5 smoothing element
// from the posterior it has just produced and folds the thread's block of
// them (Lemma 6, associativity lets the fold run forward), writing one
// smoothing block aggregate per thread to `sagg` for the reverse scan.
// With TV the elements are a time-varying model's TVElem records (`el`) and
// the fused smoothing elements use the next step's transition from `tv`.
// Shared memory of one forward tile: the model constants (single sequence)
// and the block scan's.
template <int N, int M, int NT>
struct FilterSmem {
    ModelConst<N, M> mc;
    BlockCoef<N, M> bc;   // block-fold coefficients of a single sequence
    typename BlockScan<FilterOp<N>, NT>::Smem bsm;
};

// One forward tile (`tile` of the sequence or segmented axis).  `sm.mc` holds
// the constants of a single sequence (unused by segmented scans); `dsm` is
// the staging memory of filter_dyn_smem.
template <int N, int M, int NT, int CH, bool FROM_Y, bool SAGG, bool SEG, bool TV, int REF = REF_FP64>
KS_DEV void filter_scan_body(FilterSmem<N, M, NT>& sm, char* dsm, int tile,
                             const float* __restrict__ y, const float* __restrict__ el, int64_t ld, int64_t T,
                             float* __restrict__ fmean, float* __restrict__ fcov, const ScanState& ss,
                             float* __restrict__ sagg, const Segs<N, M>& segs, const TVArgs& tv) {
    static_assert(FROM_Y || !SEG, "segmented scans build their elements from y");
    static_assert(!TV || (!FROM_Y && !SEG), "time-varying elements come materialised");
    using BS = BlockScan<FilterOp<N, REF>, NT>;
    using SG = Stage<N>;
    constexpr int64_t TILE = (int64_t)NT * CH;
    constexpr int OSTR = SG::pad_odd(SG::kBuf);
    const ModelConst<N, M>& mc = sm.mc;
    typename BS::Smem& bsm = sm.bsm;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t k0 = tile * TILE + (int64_t)tid * CH;
    const bool valid = k0 < T;
    Flags bad = 0u;

    // ---- phase 1: fold this thread's block of steps
    FElem<N> acc;
    Cursor<N, M, SEG> cur;
    if (!valid) {
        set_identity<N>(acc);
    } else if constexpr (FROM_Y) {
        cur.seek(segs, &mc, k0, T);
        // A full block inside one sequence, not holding its first step, folds
        // through the block coefficients (the linear block fold).
        const BlockCoef<N, M>* bcf = nullptr;
        if (segs.coef != nullptr) bcf = SEG ? segs.coef + cur.s : &sm.bc;
        const bool lin = bcf != nullptr && bcf->ch == CH && k0 + CH <= T && !cur.first(k0) &&
                         (!SEG || cur.end >= k0 + CH);
        if (lin) {
#pragma unroll
            for (int a = 0; a < N * N; ++a) acc.A[a] = bcf->A[a];
#pragma unroll
            for (int a = 0; a < sym_size(N); ++a) { acc.C[a] = bcf->C[a]; acc.J[a] = bcf->J[a]; }
            float y0[M];
            load_meas<M>(y, k0, y0);
#pragma unroll
            for (int a = 0; a < N; ++a) {
                float sb = bcf->bc[a], se = bcf->ec[a];
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    sb = fmaf(bcf->Bs[a * M + q], y0[q], sb);
                    se = fmaf(bcf->Es[a * M + q], y0[q], se);
                }
                acc.b[a] = sb;
                acc.eta[a] = se;
            }
#pragma unroll 4
            for (int i = 1; i < CH; ++i) {   // the other steps relative to the first
                float dy[M];
                load_meas<M>(y, k0 + i, dy);
#pragma unroll
                for (int q = 0; q < M; ++q) dy[q] -= y0[q];
#pragma unroll
                for (int a = 0; a < N; ++a)
#pragma unroll
                    for (int q = 0; q < M; ++q) {
                        acc.b[a] = fmaf(bcf->Bc[i][a * M + q], dy[q], acc.b[a]);
                        acc.eta[a] = fmaf(bcf->Ec[i][a * M + q], dy[q], acc.eta[a]);
                    }
            }
        } else {
        // y of the next step is loaded one step ahead, so that its latency
        // overlaps the current step's combine
        float yn[M];
        load_meas<M>(y, k0, yn);
        if (cur.first(k0)) {
            first_element<N, M>(*cur.mc, acc);
        } else {
            float b[N], w[M];
            meas_element<N, M>(*cur.mc, yn, b, w);
            expand_meas<N, M>(*cur.mc, b, w, acc);
        }
        if (k0 + 1 < T) load_meas<M>(y, k0 + 1, yn);
#pragma unroll 1
        for (int i = 1; i < CH; ++i) {
            const int64_t k = k0 + i;
            if (k >= T) break;
            float yk[M];
#pragma unroll
            for (int a = 0; a < M; ++a) yk[a] = yn[a];
            if (i + 1 < CH && k + 1 < T) load_meas<M>(y, k + 1, yn);
            cur.forward(segs, k);
            if (cur.first(k)) {   // acc (x) a_1 = (0, b_1, C_1, eta_acc, J_acc) since A_1 = 0, eta_1 = J_1 = 0
#pragma unroll
                for (int a = 0; a < N * N; ++a) acc.A[a] = 0.f;
#pragma unroll
                for (int a = 0; a < N; ++a) acc.b[a] = cur.mc->b1[a];
#pragma unroll
                for (int a = 0; a < sym_size(N); ++a) acc.C[a] = cur.mc->C1[a];
            } else {
                float b[N], w[M];
                meas_element<N, M>(*cur.mc, yk, b, w);
                acc = fcombine_meas<N, M>(acc, *cur.mc, b, w, bad);
            }
        }
        }
    } else if constexpr (TV) {
        TVElem<N, M> te;
        load_tvelem<N, M>(el, k0, te);
        expand_meas<N, M>(te, te.b, te.w, acc);
#pragma unroll 1
        for (int i = 1; i < CH; ++i) {
            const int64_t k = k0 + i;
            if (k >= T) break;
            load_tvelem<N, M>(el, k, te);
            acc = fcombine_meas<N, M>(acc, te, te.b, te.w, bad);
        }
    } else {
        acc = load_soa<N>(el, ld, k0);
#pragma unroll 1
        for (int i = 1; i < CH; ++i) {
            const int64_t k = k0 + i;
            if (k >= T) break;
            acc = fcombine<N>(acc, load_soa<N>(el, ld, k), bad);
        }
    }

    // ---- phase 2
    FState<N> st;
    bool has = false;
    BS::run(bsm, ss, tile, acc, st, has, bad);

    // ---- phase 3: step through the block from the incoming posterior
    if (valid) {
        char* obuf = dsm + tid * OSTR;
        int gcnt = 0;
        int64_t gk = k0;
        bool pending = false;
        float probe = 0.f;
        SElem<N> sacc;
        // Single sequence, 32 steps per thread: step k's Lemma 5 element is
        // built in the next iteration, beside the advance to step k + 1, which
        // does not depend on it (two independent chains in one loop body).
        // With 4 steps per thread the element left over after the loop costs
        // more than the overlap gains.
        constexpr bool LAG = FROM_Y && SAGG && !SEG && !TV && CH >= 32;
        int nsteps = 0;
        float yn[M];
        if constexpr (FROM_Y) {
            cur.seek(segs, &mc, k0, T);
            load_meas<M>(y, k0, yn);
        }
#pragma unroll 1
        for (int i = 0; i < CH; ++i) {
            const int64_t k = k0 + i;
            if (k >= T) break;
            const FState<N> prev = st;    // posterior of step k - 1 (i >= 1)
            if constexpr (FROM_Y) {
                float yk[M];
#pragma unroll
                for (int a = 0; a < M; ++a) yk[a] = yn[a];
                if (i + 1 < CH && k + 1 < T) load_meas<M>(y, k + 1, yn);   // one step ahead
                cur.forward(segs, k);
                if (cur.first(k)) {  // posterior (x) a_1 = (b_1, C_1): A_1 = 0
#pragma unroll
                    for (int a = 0; a < N; ++a) st.b[a] = cur.mc->b1[a];
#pragma unroll
                    for (int a = 0; a < sym_size(N); ++a) st.C[a] = cur.mc->C1[a];
                    has = true;
                } else {
                    float b[N], w[M];
                    meas_element<N, M>(*cur.mc, yk, b, w);
                    fadvance_meas<N, M>(st, *cur.mc, b, w, bad);
                }
            } else if constexpr (TV) {
                TVElem<N, M> te;
                load_tvelem<N, M>(el, k, te);
                if (!has) {   // step 0: A = 0, U = w = 0
#pragma unroll
                    for (int a = 0; a < N; ++a) st.b[a] = te.b[a];
#pragma unroll
                    for (int a = 0; a < sym_size(N); ++a) st.C[a] = te.C[a];
                    has = true;
                } else {
                    fadvance_meas<N, M>(st, te, te.b, te.w, bad);
                }
            } else {
                const FElem<N> e = load_soa<N>(el, ld, k);
                if (!has) {
                    st = FilterOp<N>::state_of(e);
                    has = true;
                } else {
                    fadvance<N>(st, e, bad);
                }
            }
            probe += finite_probe<N>(st.b, st.C);
            ++nsteps;
            if constexpr (LAG) {
                if (i >= 1) {   // step k - 1 < T - 1: never the last step
                    SElem<N> e;
                    smoother_element<N, M>(*cur.mc, prev.b, prev.C, e, bad);
                    sacc = (i == 1) ? e : scombine<N>(sacc, e);
                }
            } else if constexpr (SAGG) {
                SElem<N> e;
                if constexpr (TV) build_selem_tv<N, M>(tv, k, T, st.b, st.C, e, bad);
                else build_selem_from<N, M>(*cur.mc, st.b, st.C, cur.last(k), e, bad);
                sacc = (i == 0) ? e : scombine<N>(sacc, e);
            }
            if constexpr (SG::kOn) {
                if (gcnt == 0 && pending) bulk_wait_read_all();
                stage_write<N>(obuf, gcnt, st.b, st.C);
                ++gcnt;
                if (gcnt == SG::G || k == T - 1 || i == CH - 1) {
                    stage_flush<N>(obuf, fmean, fcov, gk, gcnt);
                    pending = true;
                    gk += gcnt;
                    gcnt = 0;
                }
            } else {
                store_posterior<N>(fmean, fcov, k, st.b, st.C);
            }
        }
        if constexpr (LAG) {   // the block's last step
            const int64_t kl = k0 + nsteps - 1;
            SElem<N> e;
            build_selem_from<N, M>(*cur.mc, st.b, st.C, kl == T - 1, e, bad);
            sacc = (nsteps == 1) ? e : scombine<N>(sacc, e);
        }
        if constexpr (SG::kOn) {
            if (pending) bulk_wait_all();
        }
        if constexpr (SAGG) store_plain(sagg + (k0 / CH) * (int64_t)(sizeof(SElem<N>) / 4), sacc);
        bad |= !isfinite(probe);
    }
    report_flags(ss.status, bad, kFull, lane == 0);
}

// REF: how the cross-block combines take their inverses.  The fused scans
// run first with REF_DETECT (FP32 inverses with a condition estimate, which
// keeps the kernel's registers for its step loops) and then launch a RETRY
// copy with REF_FP64 that returns at once unless the first run met an
// ill-conditioned inverse (HDR_NEED); then it repeats the scan with the FP64
// refinement, on its own tile counter and flags, and overwrites the results.
template <int N, int M, int NT, int CH, bool FROM_Y, bool SAGG, bool SEG, bool TV, int REF = REF_FP64,
          bool RETRY = false>
__global__ void __launch_bounds__(NT) filter_scan_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                         const float* __restrict__ y,
                                                         const float* __restrict__ el, int64_t ld,
                                                         int64_t T, float* __restrict__ fmean,
                                                         float* __restrict__ fcov, ScanState ss,
                                                         float* __restrict__ sagg, Segs<N, M> segs,
                                                         TVArgs tv) {
    pdl_wait();   // the preparation (or the first run) has completed
    if constexpr (RETRY) {
        if (*(volatile uint32_t*)(ss.status + HDR_NEED) == 0u) {   // the first run needed no refinement
            pdl_trigger();
            return;
        }
    }
    __shared__ FilterSmem<N, M, NT> sm;
    __shared__ int s_tile;
    extern __shared__ __align__(16) char dsm[];
    const int tid = threadIdx.x;
    load_const<N, M>(mcg, sm.mc, tid, NT);
    if (!SEG && segs.coef != nullptr) load_coef<N, M>(segs.coef, sm.bc, tid, NT);
    if (tid == 0) s_tile = (int)atomicAdd(ss.counter, 1u);
    __syncthreads();
    const int tile = s_tile;
    if (tile < (int)gridDim.x)   // else a tile number past the grid (only when the counter was offset)
        filter_scan_body<N, M, NT, CH, FROM_Y, SAGG, SEG, TV, REF>(sm, dsm, tile, y, el, ld, T, fmean, fcov, ss,
                                                                   sagg, segs, tv);
    pdl_trigger();
}

// ---------------------------------------------------------------- reverse scan
// Tiles and threads walk the reversed sequence r = T-1-k; in that order the
// scan operator is x (x)_r y = y (x) x (Lemma 6 with the earlier time step
// on the left), so the inclusive r-prefixes are Theorem 2's suffix sums.
// Per-thread source of filtered moments for the reverse scan: either staged
// groups of G steps fetched by bulk copies (double-buffered), or direct rows.
template <int N>
struct RevReader {
    using SG = Stage<N>;
    static constexpr int BSTR = SG::pad_odd(SG::kBuf);
    static constexpr int TSTR = 2 * BSTR + 16;      // per thread: odd number of 16-byte units
    char* base;
    uint64_t* mb;
    uint32_t par0, par1;
    int64_t khi;      // first (latest) step of the thread's block
    int cnt;          // steps in the block
    int ngroups;

    KS_DEV void init(char* b, uint64_t* mbar, int64_t k_hi, int count) {
        base = b;
        mb = mbar;
        par0 = par1 = 0u;
        khi = k_hi;
        cnt = count;
        ngroups = (count + SG::G - 1) / SG::G;
    }
    KS_DEV char* buf(int g) const { return base + (g & 1) * BSTR; }
    // group g covers steps khi - g*G down to max(khi - g*G - G + 1, khi - cnt + 1)
    KS_DEV int64_t glo(int g) const {
        const int64_t lo = khi - (int64_t)g * SG::G - SG::G + 1;
        const int64_t lim = khi - cnt + 1;
        return lo > lim ? lo : lim;
    }
    KS_DEV int gcount(int g) const { return (int)(khi - (int64_t)g * SG::G - glo(g) + 1); }
    KS_DEV void fetch(const float* fm, const float* fc, int g) {
        if (g < ngroups) stage_fetch<N>(buf(g), fm, fc, glo(g), gcount(g), mb + (g & 1));
    }
    KS_DEV bool wait(int g, uint32_t limit) {
        const bool odd = (g & 1) != 0;
        const bool ok = mbar_wait(mb + (g & 1), odd ? par1 : par0, limit);
        if (odd) par1 ^= 1u; else par0 ^= 1u;
        return ok;
    }
};

// With staged reads the reverse scan's shared memory allows two blocks per SM,
// so up to 255 registers per thread cost no occupancy and the paired element
// builds of phase 3 keep theirs; otherwise the compiler's default applies (0).
template <int N>
constexpr int kRevMinBlocks = Stage<N>::kOn ? 2 : 0;

// Blocks of CH steps start at multiples of CH from step 0 (the forward
// scan's grid); the reverse scan visits them last block first.  With FROM_AGG
// each thread's block aggregate comes from the forward scan (`sagg`);
// otherwise it is folded here from the filtered moments.
// With TV the elements come from a time-varying model's per-step transitions
// (`tv`) instead of the constant model.
// Shared memory of one reverse tile: the model constants (single sequence),
// the block scan's, and the staged reads' mbarriers (two per thread).
template <int N, int M, int NT>
struct SmootherSmem {
    ModelConst<N, M> mc;
    typename BlockScan<SmootherOp<N>, NT>::Smem bsm;
    uint64_t mbars[Stage<N>::kOn ? 2 * NT : 1];
};

// One reverse tile; the mbarriers of `sm` must be initialised (one arrival)
// and have no transaction pending, as the body leaves them.
template <int N, int M, int NT, int CH, bool FROM_AGG, bool SEG, bool TV>
KS_DEV void smoother_scan_body(SmootherSmem<N, M, NT>& sm, char* dsm, int tile,
                               const float* __restrict__ fmean, const float* __restrict__ fcov, int64_t T,
                               float* __restrict__ smean, float* __restrict__ scov, const ScanState& ss,
                               const float* __restrict__ sagg, const Segs<N, M>& segs, const TVArgs& tv) {
    static_assert(!TV || !SEG, "time-varying models run unsegmented");
    using BS = BlockScan<SmootherOp<N>, NT>;
    using SG = Stage<N>;
    using RR = RevReader<N>;
    const ModelConst<N, M>& mc = sm.mc;
    typename BS::Smem& bsm = sm.bsm;
    uint64_t* mbars = sm.mbars;
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t nblk = (T + CH - 1) / CH;
    const int64_t c = nblk - 1 - ((int64_t)tile * NT + tid);    // forward block index
    const bool valid = c >= 0;
    const int64_t klo = c * CH;
    const int64_t khi = valid ? ((klo + CH < T ? klo + CH : T) - 1) : -1;
    const int cnt = valid ? (int)(khi - klo + 1) : 0;
    Flags bad = 0u;
    bool lost = false;
    constexpr uint32_t kWait = 4000000u;
    RR rd;
    if constexpr (SG::kOn) rd.init(dsm + tid * RR::TSTR, &mbars[2 * tid], khi, cnt);

    // ---- phase 1: a_{k_lo} (x) ... (x) a_{k_hi} over this thread's steps
    SElem<N> acc;
    set_identity<N>(acc);
    if constexpr (FROM_AGG) {
        if (valid) acc = load_cg<SElem<N>>(sagg + c * (int64_t)(sizeof(SElem<N>) / 4));
    } else if (valid) {
        Cursor<N, M, SEG> cur;
        cur.seek(segs, &mc, khi, T);
        if constexpr (SG::kOn) {
            rd.fetch(fmean, fcov, 0);
            rd.fetch(fmean, fcov, 1);
            bool first = true;
#pragma unroll 1
            for (int g = 0; g < rd.ngroups; ++g) {
                lost |= !rd.wait(g, kWait);
                const int gc = rd.gcount(g);
                const int64_t lo = rd.glo(g);
#pragma unroll 1
                for (int s = gc - 1; s >= 0; --s) {
                    float xb[N], P[sym_size(N)];
                    stage_read<N>(rd.buf(g), s, xb, P);
                    cur.backward(segs, lo + s);
                    SElem<N> e;
                    if constexpr (TV) build_selem_tv<N, M>(tv, lo + s, T, xb, P, e, bad);
                    else build_selem_from<N, M>(*cur.mc, xb, P, cur.last(lo + s), e, bad);
                    acc = first ? e : scombine<N>(e, acc);
                    first = false;
                }
                rd.fetch(fmean, fcov, g + 2);
            }
        } else {
#pragma unroll 1
            for (int i = 0; i < cnt; ++i) {
                const int64_t k = khi - i;
                float xb[N], P[sym_size(N)];
                load_posterior<N>(fmean, fcov, k, xb, P);
                cur.backward(segs, k);
                SElem<N> e;
                if constexpr (TV) build_selem_tv<N, M>(tv, k, T, xb, P, e, bad);
                else build_selem_from<N, M>(*cur.mc, xb, P, cur.last(k), e, bad);
                acc = (i == 0) ? e : scombine<N>(e, acc);
            }
        }
    }

    // ---- phase 2
    SState<N> st;
    bool has = false;
    BS::run(bsm, ss, tile, acc, st, has, bad);

    // ---- phase 3
    if (valid) {
        float probe = 0.f;
        Cursor<N, M, SEG> cur;
        cur.seek(segs, &mc, khi, T);
        if constexpr (SG::kOn) {
            rd.fetch(fmean, fcov, 0);
            rd.fetch(fmean, fcov, 1);
#pragma unroll 1
            for (int g = 0; g < rd.ngroups; ++g) {
                lost |= !rd.wait(g, kWait);
                const int gc = rd.gcount(g);
                const int64_t lo = rd.glo(g);
                char* b = rd.buf(g);
                int s = gc - 1;
                // The next group's moments go into the buffer that the store
                // of the previous group reads; that store was issued a whole
                // group ago, so the refill waits for it after this group's
                // first steps rather than right after issuing a store.
                bool refill = (g >= 1) && (g + 1 < rd.ngroups);
                // Two steps at a time: a step's Lemma 5 element depends only on
                // its filtered moments, not on the running smoothed state, so
                // the two element builds run side by side and only the two
                // applications form the chain.
#pragma unroll 1
                for (; s >= 1; s -= 2) {
                    float xa[N], Pa[sym_size(N)], xc[N], Pc[sym_size(N)];
                    stage_read<N>(b, s, xa, Pa);     // later step
                    stage_read<N>(b, s - 1, xc, Pc);
                    const int64_t ka = lo + s, kc = ka - 1;
                    cur.backward(segs, ka);
                    const ModelConst<N, M>* ma = cur.mc;
                    const bool la = TV ? (ka == T - 1) : cur.last(ka);
                    cur.backward(segs, kc);
                    const ModelConst<N, M>* mcc = cur.mc;
                    const bool lc = TV ? (kc == T - 1) : cur.last(kc);
                    SElem<N> ea, ec;
                    build_selem_flat<N, M, TV>(ma, tv, ka, T, la, xa, Pa, ea, bad);
                    build_selem_flat<N, M, TV>(mcc, tv, kc, T, lc, xc, Pc, ec, bad);
                    if (!has) { st = SmootherOp<N>::state_of(ea); has = true; }   // only k = T-1
                    else sadvance<N>(ea, st);
                    stage_write<N>(b, s, st.g, st.L);     // the slot's input is already in registers
                    probe += finite_probe<N>(st.g, st.L);
                    sadvance<N>(ec, st);                  // a segment's last step has E = 0
                    stage_write<N>(b, s - 1, st.g, st.L);
                    probe += finite_probe<N>(st.g, st.L);
                    if (refill) {
                        bulk_wait_read_all();
                        rd.fetch(fmean, fcov, g + 1);
                        refill = false;
                    }
                }
                if (s == 0) {
                    float xb[N], P[sym_size(N)];
                    stage_read<N>(b, 0, xb, P);
                    cur.backward(segs, lo);
                    SElem<N> e;
                    if constexpr (TV) build_selem_tv<N, M>(tv, lo, T, xb, P, e, bad);
                    else build_selem_from<N, M>(*cur.mc, xb, P, cur.last(lo), e, bad);
                    if (!has) { st = SmootherOp<N>::state_of(e); has = true; }
                    else sadvance<N>(e, st);
                    stage_write<N>(b, 0, st.g, st.L);
                    probe += finite_probe<N>(st.g, st.L);
                }
                if (refill) {
                    bulk_wait_read_all();
                    rd.fetch(fmean, fcov, g + 1);
                }
                stage_flush<N>(b, smean, scov, lo, gc);
            }
            bulk_wait_all();
        } else {
#pragma unroll 1
            for (int i = 0; i < cnt; ++i) {
                const int64_t k = khi - i;
                float xb[N], P[sym_size(N)];
                load_posterior<N>(fmean, fcov, k, xb, P);
                cur.backward(segs, k);
                SElem<N> e;
                if constexpr (TV) build_selem_tv<N, M>(tv, k, T, xb, P, e, bad);
                else build_selem_from<N, M>(*cur.mc, xb, P, cur.last(k), e, bad);
                if (!has) { st = SmootherOp<N>::state_of(e); has = true; }
                else sadvance<N>(e, st);
                store_posterior<N>(smean, scov, k, st.g, st.L);
                probe += finite_probe<N>(st.g, st.L);
            }
        }
        bad |= !isfinite(probe);
    }
    if (lost) atomicOr(ss.status, ST_TIMEOUT);
    report_flags(ss.status, bad, kFull, lane == 0);
}

template <int N, int M, int NT, int CH, bool FROM_AGG, bool SEG, bool TV>
__global__ void __launch_bounds__(NT, kRevMinBlocks<N>) smoother_scan_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                           const float* __restrict__ fmean,
                                                           const float* __restrict__ fcov, int64_t T,
                                                           float* __restrict__ smean,
                                                           float* __restrict__ scov, ScanState ss,
                                                           const float* __restrict__ sagg, Segs<N, M> segs,
                                                           TVArgs tv) {
    __shared__ SmootherSmem<N, M, NT> sm;
    __shared__ int s_tile;
    extern __shared__ __align__(16) char dsm[];
    const int tid = threadIdx.x;
    pdl_wait();   // the forward scan has completed
    load_const<N, M>(mcg, sm.mc, tid, NT);
    if (tid == 0) s_tile = (int)atomicAdd(ss.counter, 1u);
    if constexpr (Stage<N>::kOn) {
        mbar_init(&sm.mbars[2 * tid], 1);
        mbar_init(&sm.mbars[2 * tid + 1], 1);
        fence_proxy_async();
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile >= (int)gridDim.x) return;   // a tile number past the grid (only when the counter was offset)
    smoother_scan_body<N, M, NT, CH, FROM_AGG, SEG, TV>(sm, dsm, tile, fmean, fcov, T, smean, scov, ss, sagg, segs,
                                                        tv);
    pdl_trigger();
}

// Dynamic shared memory of the two scans (bytes).
template <int N, int NT>
constexpr int filter_dyn_smem() {
    return Stage<N>::kOn ? NT * Stage<N>::pad_odd(Stage<N>::kBuf) : 16;
}
template <int N, int NT>
constexpr int smoother_dyn_smem() {
    return Stage<N>::kOn ? NT * RevReader<N>::TSTR : 16;
}

// ---------------------------------------------------------------- operator batches
template <int N>
KS_DEV FElem<N> load_packed_f(const float* __restrict__ p) {
    FElem<N> e;
#pragma unroll
    for (int a = 0; a < N * N; ++a) e.A[a] = p[a];
#pragma unroll
    for (int a = 0; a < N; ++a) { e.b[a] = p[N * N + a]; e.eta[a] = p[2 * N * N + N + a]; }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            e.C[sidx(a, b)] = 0.5f * (p[N * N + N + a * N + b] + p[N * N + N + b * N + a]);
            e.J[sidx(a, b)] = 0.5f * (p[2 * N * N + 2 * N + a * N + b] + p[2 * N * N + 2 * N + b * N + a]);
        }
    return e;
}

template <int N>
__global__ void filter_combine_batch_kernel(const float* __restrict__ left, const float* __restrict__ right,
                                            float* __restrict__ out, int64_t count, uint32_t* status) {
    constexpr int SZ = 3 * N * N + 2 * N;
    Flags bad = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const FElem<N> r = fcombine<N>(load_packed_f<N>(left + i * SZ), load_packed_f<N>(right + i * SZ), bad);
        float* o = out + i * SZ;
#pragma unroll
        for (int a = 0; a < N * N; ++a) o[a] = r.A[a];
#pragma unroll
        for (int a = 0; a < N; ++a) { o[N * N + a] = r.b[a]; o[2 * N * N + N + a] = r.eta[a]; }
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b < N; ++b) {
                o[N * N + N + a * N + b] = r.C[sidx(a, b)];
                o[2 * N * N + 2 * N + a * N + b] = r.J[sidx(a, b)];
            }
    }
    if (bad & FL_BAD) atomicOr(status, ST_NUMERIC);
}

template <int N>
__global__ void smoother_combine_batch_kernel(const float* __restrict__ left, const float* __restrict__ right,
                                              float* __restrict__ out, int64_t count) {
    constexpr int SZ = 2 * N * N + N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        SElem<N> l, r;
        const float* pl = left + i * SZ;
        const float* pr = right + i * SZ;
#pragma unroll
        for (int a = 0; a < N * N; ++a) { l.E[a] = pl[a]; r.E[a] = pr[a]; }
#pragma unroll
        for (int a = 0; a < N; ++a) { l.g[a] = pl[N * N + a]; r.g[a] = pr[N * N + a]; }
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) {
                l.L[sidx(a, b)] = 0.5f * (pl[N * N + N + a * N + b] + pl[N * N + N + b * N + a]);
                r.L[sidx(a, b)] = 0.5f * (pr[N * N + N + a * N + b] + pr[N * N + N + b * N + a]);
            }
        const SElem<N> c = scombine<N>(l, r);
        float* o = out + i * SZ;
#pragma unroll
        for (int a = 0; a < N * N; ++a) o[a] = c.E[a];
#pragma unroll
        for (int a = 0; a < N; ++a) o[N * N + a] = c.g[a];
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b < N; ++b) o[N * N + N + a * N + b] = c.L[sidx(a, b)];
    }
}

}  // namespace ks
