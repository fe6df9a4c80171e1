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

#include "ks_ops.cuh"

namespace ks {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kFlagAgg = 1u;   // tile aggregate published
constexpr uint32_t kFlagPre = 2u;   // inclusive prefix published

struct ScanState {
    uint32_t* counter;   // tile counter (zeroed before launch)
    uint32_t* flags;     // per-tile flags (zeroed before launch)
    float* agg;          // per-tile aggregates
    float* pre;          // per-tile inclusive prefixes
    uint32_t* status;    // device status word
    uint32_t spin_limit; // look-back polls before giving up (~1 s)
};

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
KS_DEV void load_const(const ModelConst<N, M>* __restrict__ g, ModelConst<N, M>& s, int tid, int nt) {
    const float* src = reinterpret_cast<const float*>(g);
    float* dst = reinterpret_cast<float*>(&s);
    for (int i = tid; i < (int)(sizeof(ModelConst<N, M>) / 4); i += nt) dst[i] = __ldg(src + i);
}

// ---------------------------------------------------------------- prep
// Model constants.  k > 1 quantities in FP32 (Lemma 3 with the Cholesky
// factor of S); the k = 1 element (Kalman prediction and update from
// N(m0, P0), Lemma 3) in FP64.  One thread: the work is O(N^3).
template <int N, int M>
__global__ void prep_kernel(const float* __restrict__ F, const float* __restrict__ u,
                            const float* __restrict__ Q, const float* __restrict__ H,
                            const float* __restrict__ d, const float* __restrict__ R,
                            const double* __restrict__ m0, const double* __restrict__ P0,
                            const float* __restrict__ y, ModelConst<N, M>* __restrict__ out,
                            uint32_t* __restrict__ status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    ModelConst<N, M> mc;
    bool ok = true;
    float Hm[M][N], Fm[N][N], Qs[N][N], Rs[M][M], uv[N], dv[M];
    for (int a = 0; a < N; ++a) {
        uv[a] = u ? u[a] : 0.f;
        for (int b = 0; b < N; ++b) { Fm[a][b] = F[a * N + b]; Qs[a][b] = Q[a * N + b]; }
    }
    for (int q = 0; q < M; ++q) {
        dv[q] = d ? d[q] : 0.f;
        for (int a = 0; a < N; ++a) Hm[q][a] = H[q * N + a];
        for (int p = 0; p < M; ++p) Rs[q][p] = R[q * M + p];
    }
    for (int a = 0; a < N; ++a) {
        mc.u[a] = uv[a];
        for (int b = 0; b < N; ++b) mc.F[a * N + b] = Fm[a][b];
        for (int b = 0; b <= a; ++b) mc.Q[sidx(a, b)] = 0.5f * (Qs[a][b] + Qs[b][a]);
    }
    // S = H Q H^T + R, S = Ls Ls^T, Lsi = Ls^{-1}
    float HQ[M][N], S[M][M], Ls[M][M], Lsi[M][M];
    for (int q = 0; q < M; ++q)
        for (int a = 0; a < N; ++a) {
            float s = 0.f;
            for (int c = 0; c < N; ++c) s = fmaf(Hm[q][c], mc.Q[sidx(c, a)], s);
            HQ[q][a] = s;
        }
    for (int q = 0; q < M; ++q)
        for (int p = 0; p < M; ++p) {
            float s = 0.5f * (Rs[q][p] + Rs[p][q]);
            for (int c = 0; c < N; ++c) s = fmaf(HQ[q][c], Hm[p][c], s);
            S[q][p] = s;
        }
    for (int j = 0; j < M; ++j) {
        float s = S[j][j];
        for (int l = 0; l < j; ++l) s -= Ls[j][l] * Ls[j][l];
        ok = ok && (s > 0.f);
        Ls[j][j] = sqrtf(fmaxf(s, 1e-37f));
        for (int i = j + 1; i < M; ++i) {
            float t = S[i][j];
            for (int l = 0; l < j; ++l) t -= Ls[i][l] * Ls[j][l];
            Ls[i][j] = t / Ls[j][j];
        }
        for (int i = 0; i < j; ++i) Ls[i][j] = 0.f;
    }
    for (int c = 0; c < M; ++c)
        for (int i = 0; i < M; ++i) {
            if (i < c) { Lsi[i][c] = 0.f; continue; }
            float t = (i == c) ? 1.f : 0.f;
            for (int l = c; l < i; ++l) t -= Ls[i][l] * Lsi[l][c];
            Lsi[i][c] = t / Ls[i][i];
        }
    // tmp = Lsi H Q  (so K = tmp^T Lsi and K S K^T = tmp^T tmp)
    float tmp[M][N], HF[M][N];
    for (int q = 0; q < M; ++q)
        for (int a = 0; a < N; ++a) {
            float s = 0.f, h = 0.f;
            for (int p = 0; p <= q; ++p) s = fmaf(Lsi[q][p], HQ[p][a], s);
            for (int c = 0; c < N; ++c) h = fmaf(Hm[q][c], Fm[c][a], h);
            tmp[q][a] = s;
            HF[q][a] = h;
        }
    float K[N][M];
    for (int a = 0; a < N; ++a)
        for (int q = 0; q < M; ++q) {
            float s = 0.f;
            for (int p = q; p < M; ++p) s = fmaf(tmp[p][a], Lsi[p][q], s);
            K[a][q] = s;
            mc.K[a * M + q] = s;
        }
    for (int q = 0; q < M; ++q) {
        for (int p = 0; p < M; ++p) mc.Lsi[q * M + p] = Lsi[q][p];
        float s = dv[q];
        for (int c = 0; c < N; ++c) s = fmaf(Hm[q][c], uv[c], s);
        mc.hud[q] = s;
        for (int a = 0; a < N; ++a) {
            float t = 0.f;
            for (int p = 0; p <= q; ++p) t = fmaf(Lsi[q][p], HF[p][a], t);
            mc.U[q * N + a] = t;
        }
    }
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            float s = Fm[a][b];
            for (int q = 0; q < M; ++q) s = fmaf(-K[a][q], HF[q][b], s);
            mc.A[a * N + b] = s;
        }
    for (int a = 0; a < N; ++a)
        for (int b = 0; b <= a; ++b) {
            float s = mc.Q[sidx(a, b)];
            for (int q = 0; q < M; ++q) s = fmaf(-tmp[q][a], tmp[q][b], s);
            mc.C[sidx(a, b)] = s;
        }
    // ---- k = 1 in FP64: m- = F m0 + u, P- = F P0 F^T + Q, S1 = H P- H^T + R,
    //      K1 = P- H^T S1^{-1}, b1 = m- + K1 (y1 - H m- - d), C1 = P- - K1 S1 K1^T
    //      (skipped when no measurements are given: the smoother needs none of it)
    for (int a = 0; a < N; ++a) mc.b1[a] = 0.f;
    for (int a = 0; a < sym_size(N); ++a) mc.C1[a] = 0.f;
    if (y != nullptr) {
        double mm[N], FP[N][N], Pm[N][N], HP[M][N], S1[M][M], L1[M][M], t1[M][N], e1[M], z[M];
        for (int a = 0; a < N; ++a) {
            double s = uv[a];
            for (int c = 0; c < N; ++c) s += (double)Fm[a][c] * m0[c];
            mm[a] = s;
        }
        for (int a = 0; a < N; ++a)
            for (int b = 0; b < N; ++b) {
                double s = 0.0;
                for (int c = 0; c < N; ++c) s += (double)Fm[a][c] * P0[c * N + b];
                FP[a][b] = s;
            }
        for (int a = 0; a < N; ++a)
            for (int b = 0; b < N; ++b) {
                double s = 0.5 * ((double)Qs[a][b] + (double)Qs[b][a]);
                for (int c = 0; c < N; ++c) s += FP[a][c] * (double)Fm[b][c];
                Pm[a][b] = s;
            }
        for (int q = 0; q < M; ++q)
            for (int a = 0; a < N; ++a) {
                double s = 0.0;
                for (int c = 0; c < N; ++c) s += (double)Hm[q][c] * Pm[c][a];
                HP[q][a] = s;
            }
        for (int q = 0; q < M; ++q)
            for (int p = 0; p < M; ++p) {
                double s = 0.5 * ((double)Rs[q][p] + (double)Rs[p][q]);
                for (int c = 0; c < N; ++c) s += HP[q][c] * (double)Hm[p][c];
                S1[q][p] = s;
            }
        for (int j = 0; j < M; ++j) {
            double s = S1[j][j];
            for (int l = 0; l < j; ++l) s -= L1[j][l] * L1[j][l];
            ok = ok && (s > 0.0);
            L1[j][j] = sqrt(s > 0.0 ? s : 1e-300);
            for (int i = j + 1; i < M; ++i) {
                double t = S1[i][j];
                for (int l = 0; l < j; ++l) t -= L1[i][l] * L1[j][l];
                L1[i][j] = t / L1[j][j];
            }
        }
        // t1 = L1^{-1} H P-  (K1 S1 K1^T = t1^T t1),  z = L1^{-1} e1
        for (int a = 0; a < N; ++a)
            for (int q = 0; q < M; ++q) {
                double t = HP[q][a];
                for (int l = 0; l < q; ++l) t -= L1[q][l] * t1[l][a];
                t1[q][a] = t / L1[q][q];
            }
        for (int q = 0; q < M; ++q) {
            double s = (double)y[q] - (double)dv[q];
            for (int c = 0; c < N; ++c) s -= (double)Hm[q][c] * mm[c];
            e1[q] = s;
        }
        for (int q = 0; q < M; ++q) {
            double t = e1[q];
            for (int l = 0; l < q; ++l) t -= L1[q][l] * z[l];
            z[q] = t / L1[q][q];
        }
        // b1 = m- + K1 e1 = m- + t1^T z   (K1 = t1^T L1^{-1})
        for (int a = 0; a < N; ++a) {
            double s = mm[a];
            for (int q = 0; q < M; ++q) s += t1[q][a] * z[q];
            mc.b1[a] = (float)s;
        }
        for (int a = 0; a < N; ++a)
            for (int b = 0; b <= a; ++b) {
                double s = 0.5 * (Pm[a][b] + Pm[b][a]);
                for (int q = 0; q < M; ++q) s -= t1[q][a] * t1[q][b];
                mc.C1[sidx(a, b)] = (float)s;
            }
    }
    for (int i = 0; i < 4; ++i) mc.pad[i] = 0.f;
    *out = mc;
    if (!ok) atomicOr(status, ST_NUMERIC);
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

// ---------------------------------------------------------------- forward scan
template <int N, int M, int NT, int CH, bool FROM_Y>
__global__ void __launch_bounds__(NT) filter_scan_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                         const float* __restrict__ y,
                                                         const float* __restrict__ el, int64_t ld,
                                                         int64_t T, float* __restrict__ fmean,
                                                         float* __restrict__ fcov, ScanState ss) {
    constexpr int NW = NT / 32;
    constexpr int64_t TILE = (int64_t)NT * CH;
    __shared__ ModelConst<N, M> mc;
    __shared__ FElem<N> wtot[NW];
    __shared__ FState<N> texcl;
    __shared__ int s_tile, s_has;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    load_const<N, M>(mcg, mc, tid, NT);
    if (tid == 0) s_tile = (int)atomicAdd(ss.counter, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int64_t k0 = tile * TILE + (int64_t)tid * CH;
    const bool valid = k0 < T;
    bool bad = false;

    // ---- phase 1: fold this thread's block of steps
    FElem<N> acc;
    if (!valid) {
        set_identity<N>(acc);
    } else if constexpr (FROM_Y) {
        if (k0 == 0) {
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
    } else {
        acc = load_soa<N>(el, ld, k0);
#pragma unroll 1
        for (int i = 1; i < CH; ++i) {
            const int64_t k = k0 + i;
            if (k >= T) break;
            acc = fcombine<N>(acc, load_soa<N>(el, ld, k), bad);
        }
    }

    // ---- phase 2: warp scan, warp-total scan, look-back
    FElem<N> incl = acc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        FElem<N> o = shfl_up_t(incl, d);
        if (lane >= d) incl = fcombine<N>(o, incl, bad);
    }
    const FElem<N> lane_excl = shfl_up_t(incl, 1);
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    FElem<N> wpre;
    if (warp > 0) {
        wpre = wtot[0];
        for (int w = 1; w < warp; ++w) wpre = fcombine<N>(wpre, wtot[w], bad);
    }
    if (tid == NT - 1) {
        FElem<N> tagg = (NW > 1) ? fcombine<N>(wpre, wtot[NW - 1], bad) : wtot[0];
        FState<N> ex;
        int has = 0;
        constexpr int AF = sizeof(FElem<N>) / 4, PF = sizeof(FState<N>) / 4;
        if (tile == 0) {
            FState<N> inc;
#pragma unroll
            for (int a = 0; a < N; ++a) inc.b[a] = tagg.b[a];
#pragma unroll
            for (int a = 0; a < sym_size(N); ++a) inc.C[a] = tagg.C[a];
            store_plain(ss.pre, inc);
            st_release(ss.flags, kFlagPre);
#pragma unroll
            for (int a = 0; a < N; ++a) ex.b[a] = 0.f;
#pragma unroll
            for (int a = 0; a < sym_size(N); ++a) ex.C[a] = 0.f;
        } else {
            store_plain(ss.agg + (int64_t)tile * AF, tagg);
            st_release(ss.flags + tile, kFlagAgg);
            FElem<N> run;
            bool have_run = false;
            int j = tile - 1;
            while (true) {
                const uint32_t f = wait_flag(ss.flags + j, ss.spin_limit);
                if (f == 0u) {
                    atomicOr(ss.status, ST_TIMEOUT);
#pragma unroll
                    for (int a = 0; a < N; ++a) ex.b[a] = 0.f;
#pragma unroll
                    for (int a = 0; a < sym_size(N); ++a) ex.C[a] = 0.f;
                    break;
                }
                if (f == kFlagPre) {
                    ex = load_cg<FState<N>>(ss.pre + (int64_t)j * PF);
                    if (have_run) fadvance<N>(ex, run, bad);
                    break;
                }
                const FElem<N> a = load_cg<FElem<N>>(ss.agg + (int64_t)j * AF);
                run = have_run ? fcombine<N>(a, run, bad) : a;
                have_run = true;
                --j;
            }
            has = 1;
            FState<N> inc = ex;
            fadvance<N>(inc, tagg, bad);
            store_plain(ss.pre + (int64_t)tile * PF, inc);
            st_release(ss.flags + tile, kFlagPre);
        }
        texcl = ex;
        s_has = has;
    }
    __syncthreads();

    // ---- phase 3: prefix entering this thread's block, then step by step
    if (valid) {
        FState<N> st = texcl;
        bool has = s_has != 0;
        if (warp > 0) {
            if (has) {
                fadvance<N>(st, wpre, bad);
            } else {
#pragma unroll
                for (int a = 0; a < N; ++a) st.b[a] = wpre.b[a];
#pragma unroll
                for (int a = 0; a < sym_size(N); ++a) st.C[a] = wpre.C[a];
                has = true;
            }
        }
        if (lane > 0) {
            if (has) {
                fadvance<N>(st, lane_excl, bad);
            } else {
#pragma unroll
                for (int a = 0; a < N; ++a) st.b[a] = lane_excl.b[a];
#pragma unroll
                for (int a = 0; a < sym_size(N); ++a) st.C[a] = lane_excl.C[a];
                has = true;
            }
        }
        float probe = 0.f;
#pragma unroll 1
        for (int i = 0; i < CH; ++i) {
            const int64_t k = k0 + i;
            if (k >= T) break;
            if constexpr (FROM_Y) {
                if (!has) {  // only step k = 0: the first element has A_1 = 0
#pragma unroll
                    for (int a = 0; a < N; ++a) st.b[a] = mc.b1[a];
#pragma unroll
                    for (int a = 0; a < sym_size(N); ++a) st.C[a] = mc.C1[a];
                    has = true;
                } else {
                    float yk[M], b[N], w[M];
                    load_meas<M>(y, k, yk);
                    meas_element<N, M>(mc, yk, b, w);
                    fadvance_meas<N, M>(st, mc, b, w, bad);
                }
            } else {
                const FElem<N> e = load_soa<N>(el, ld, k);
                if (!has) {
#pragma unroll
                    for (int a = 0; a < N; ++a) st.b[a] = e.b[a];
#pragma unroll
                    for (int a = 0; a < sym_size(N); ++a) st.C[a] = e.C[a];
                    has = true;
                } else {
                    fadvance<N>(st, e, bad);
                }
            }
            store_posterior<N>(fmean, fcov, k, st.b, st.C);
            probe += finite_probe<N>(st.b, st.C);
        }
        bad |= !isfinite(probe);
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(ss.status, ST_NUMERIC);
}

// ---------------------------------------------------------------- reverse scan
// Tiles and threads walk the reversed sequence r = T-1-k; in that order the
// scan operator is x (x)_r y = y (x) x (Lemma 6 with the earlier time step
// on the left), so the inclusive r-prefixes are Theorem 2's suffix sums.
template <int N, int M>
KS_DEV void build_selem(const ModelConst<N, M>& mc, const float* __restrict__ fmean,
                        const float* __restrict__ fcov, int64_t T, int64_t k, SElem<N>& e, bool& bad) {
    float xb[N], P[sym_size(N)];
    load_posterior<N>(fmean, fcov, k, xb, P);
    if (k == T - 1) {  // Lemma 5, k = n: E = 0, g = xbar_n, L = P_n
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

template <int N, int M, int NT, int CH>
__global__ void __launch_bounds__(NT) smoother_scan_kernel(const ModelConst<N, M>* __restrict__ mcg,
                                                           const float* __restrict__ fmean,
                                                           const float* __restrict__ fcov, int64_t T,
                                                           float* __restrict__ smean,
                                                           float* __restrict__ scov, ScanState ss) {
    constexpr int NW = NT / 32;
    constexpr int64_t TILE = (int64_t)NT * CH;
    __shared__ ModelConst<N, M> mc;
    __shared__ SElem<N> wtot[NW];
    __shared__ SState<N> texcl;
    __shared__ int s_tile, s_has;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    load_const<N, M>(mcg, mc, tid, NT);
    if (tid == 0) s_tile = (int)atomicAdd(ss.counter, 1u);
    __syncthreads();
    const int tile = s_tile;
    const int64_t r0 = tile * TILE + (int64_t)tid * CH;
    const bool valid = r0 < T;
    bool bad = false;

    // ---- phase 1: a_{k_lo} (x) ... (x) a_{k_hi} over this thread's steps
    SElem<N> acc;
    if (!valid) {
        set_identity<N>(acc);
    } else {
        build_selem<N, M>(mc, fmean, fcov, T, T - 1 - r0, acc, bad);
#pragma unroll 1
        for (int i = 1; i < CH; ++i) {
            const int64_t r = r0 + i;
            if (r >= T) break;
            SElem<N> e;
            build_selem<N, M>(mc, fmean, fcov, T, T - 1 - r, e, bad);
            acc = scombine<N>(e, acc);
        }
    }

    // ---- phase 2
    SElem<N> incl = acc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        SElem<N> o = shfl_up_t(incl, d);
        if (lane >= d) incl = scombine<N>(incl, o);
    }
    const SElem<N> lane_excl = shfl_up_t(incl, 1);
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    SElem<N> wpre;
    if (warp > 0) {
        wpre = wtot[0];
        for (int w = 1; w < warp; ++w) wpre = scombine<N>(wtot[w], wpre);
    }
    if (tid == NT - 1) {
        SElem<N> tagg = (NW > 1) ? scombine<N>(wtot[NW - 1], wpre) : wtot[0];
        SState<N> ex;
        int has = 0;
        constexpr int AF = sizeof(SElem<N>) / 4, PF = sizeof(SState<N>) / 4;
        if (tile == 0) {
            SState<N> inc;
#pragma unroll
            for (int a = 0; a < N; ++a) inc.g[a] = tagg.g[a];
#pragma unroll
            for (int a = 0; a < sym_size(N); ++a) inc.L[a] = tagg.L[a];
            store_plain(ss.pre, inc);
            st_release(ss.flags, kFlagPre);
#pragma unroll
            for (int a = 0; a < N; ++a) ex.g[a] = 0.f;
#pragma unroll
            for (int a = 0; a < sym_size(N); ++a) ex.L[a] = 0.f;
        } else {
            store_plain(ss.agg + (int64_t)tile * AF, tagg);
            st_release(ss.flags + tile, kFlagAgg);
            SElem<N> run;
            bool have_run = false;
            int j = tile - 1;
            while (true) {
                const uint32_t f = wait_flag(ss.flags + j, ss.spin_limit);
                if (f == 0u) {
                    atomicOr(ss.status, ST_TIMEOUT);
#pragma unroll
                    for (int a = 0; a < N; ++a) ex.g[a] = 0.f;
#pragma unroll
                    for (int a = 0; a < sym_size(N); ++a) ex.L[a] = 0.f;
                    break;
                }
                if (f == kFlagPre) {
                    ex = load_cg<SState<N>>(ss.pre + (int64_t)j * PF);
                    if (have_run) sadvance<N>(run, ex);
                    break;
                }
                const SElem<N> a = load_cg<SElem<N>>(ss.agg + (int64_t)j * AF);
                run = have_run ? scombine<N>(run, a) : a;
                have_run = true;
                --j;
            }
            has = 1;
            SState<N> inc = ex;
            sadvance<N>(tagg, inc);
            store_plain(ss.pre + (int64_t)tile * PF, inc);
            st_release(ss.flags + tile, kFlagPre);
        }
        texcl = ex;
        s_has = has;
    }
    __syncthreads();

    // ---- phase 3
    if (valid) {
        SState<N> st = texcl;
        bool has = s_has != 0;
        if (warp > 0) {
            if (has) {
                sadvance<N>(wpre, st);
            } else {
#pragma unroll
                for (int a = 0; a < N; ++a) st.g[a] = wpre.g[a];
#pragma unroll
                for (int a = 0; a < sym_size(N); ++a) st.L[a] = wpre.L[a];
                has = true;
            }
        }
        if (lane > 0) {
            if (has) {
                sadvance<N>(lane_excl, st);
            } else {
#pragma unroll
                for (int a = 0; a < N; ++a) st.g[a] = lane_excl.g[a];
#pragma unroll
                for (int a = 0; a < sym_size(N); ++a) st.L[a] = lane_excl.L[a];
                has = true;
            }
        }
        float probe = 0.f;
#pragma unroll 1
        for (int i = 0; i < CH; ++i) {
            const int64_t r = r0 + i;
            if (r >= T) break;
            const int64_t k = T - 1 - r;
            SElem<N> e;
            build_selem<N, M>(mc, fmean, fcov, T, k, e, bad);
            if (!has) {  // only k = T-1: E_n = 0
#pragma unroll
                for (int a = 0; a < N; ++a) st.g[a] = e.g[a];
#pragma unroll
                for (int a = 0; a < sym_size(N); ++a) st.L[a] = e.L[a];
                has = true;
            } else {
                sadvance<N>(e, st);
            }
            store_posterior<N>(smean, scov, k, st.g, st.L);
            probe += finite_probe<N>(st.g, st.L);
        }
        bad |= !isfinite(probe);
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicOr(ss.status, ST_NUMERIC);
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
    bool bad = false;
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
    if (bad) atomicOr(status, ST_NUMERIC);
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
