// ks_hmm.cuh -- the discrete-state (hidden Markov model) instance of the
// general parallel filter and smoother of Section III: Definitions 1 and 2
// with every integral a sum over the K states (Section VI's counting measure).
//
// Model: x_0 ~ pi, p(x_k = j | x_k-1 = i) = Pi[i][j], and the measurements
// enter only through their likelihoods lik[k][j] = p(y_k | x_k = j) (0-based
// k here; step k + 1 of the paper).
//
// Elements, each thread holding whole elements in registers (K <= 8):
//  * filtering element (f, g) of Definition 1: f row-stochastic,
//    f[z*K + x] = f(x | z), and g kept as lg[z] = log g(z), so that the
//    marginal likelihoods p(y_1:k) (Theorem 1) survive long prefixes;
//  * smoothing element a of Definition 2: a[z*K + x] = a(x | z),
//    row-stochastic.
// The prefix of the filtering scan from step 1 has identical rows
// p(x_k | y_1:k) and a constant g = p(y_1:k) (Theorem 1), so it is carried
// as the state (p, L = log p(y_1:k)); the suffix of the smoothing scan to
// step n has identical rows p(x_k | y_1:n) (Theorem 2), carried as s.
//
// The per-step elements are never stored: with the likelihood row scaled to
// a maximum of 1 (its log maximum added to lg), the step-k element is
//   f_k(x | z) = Pi[z][x] l(x) / c(z),  c(z) = sum_x Pi[z][x] l(x),  g_k = c,
// and folding it into a running aggregate (f, lg) is
//   f'(x | z) = (f Pi)[z][x] l(x) / r(z),  r(z) = sum_x (f Pi)[z][x] l(x),
//   lg'(z) = lg(z) + log r(z) + log max lik[k]
// (Definition 1 with g_k f_k = Pi diag(l)).  Smoothing elements
//   a_k(x | z) = p_k(x) Pi[x][z] / sum_x' p_k(x') Pi[x'][z]
// are built from each filtered marginal p_k as the forward scan produces it.
#pragma once

#include "ks_scan.cuh"

namespace ks {
namespace hmm {

// Each element and state is padded to an odd number of floats, so that the
// block scan's per-thread shared-memory copies (one element per thread,
// thread-contiguous) fall in distinct banks.
template <int K>
struct FE {
    float f[K * K];
    float lg[K];
    float pad[(K * K + K) % 2 == 0 ? 1 : 0];
};
template <int K>
struct FS {
    float p[K];
    float L;
    float pad[(K + 1) % 2 == 0 ? 1 : 0];
};
template <int K>
struct SE {
    float a[K * K];
    float pad[(K * K) % 2 == 0 ? 1 : 0];
};
template <int K>
struct SS {
    float s[K];
    float pad[K % 2 == 0 ? 1 : 0];
};

// Model constants: the transition matrix, its transpose and the prior
// predicted to step 1 (16-byte aligned: rows are read as float4).
template <int K>
struct alignas(16) Const {
    float Pi[K * K];
    float PiT[K * K];
    float q1[K];   // p(x_1) = (pi Pi)
    float pad[(4 - K % 4) % 4];
};

// Row r of a K x K shared-memory matrix into registers (float4 when K % 4 == 0).
template <int K>
KS_DEV void load_row(const float* __restrict__ M, int r, float (&v)[K]) {
    if constexpr (K % 4 == 0) {
        const float4* p = reinterpret_cast<const float4*>(M + r * K);
#pragma unroll
        for (int i = 0; i < K / 4; ++i) {
            const float4 q = p[i];
            v[4 * i] = q.x;
            v[4 * i + 1] = q.y;
            v[4 * i + 2] = q.z;
            v[4 * i + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < K; ++i) v[i] = M[r * K + i];
    }
}

template <int K>
KS_DEV void set_identity(FE<K>& e) {
#pragma unroll
    for (int z = 0; z < K; ++z) {
#pragma unroll
        for (int x = 0; x < K; ++x) e.f[z * K + x] = (z == x) ? 1.f : 0.f;
        e.lg[z] = 0.f;
    }
}

template <int K>
KS_DEV void set_identity(SE<K>& e) {
#pragma unroll
    for (int z = 0; z < K; ++z)
#pragma unroll
        for (int x = 0; x < K; ++x) e.a[z * K + x] = (z == x) ? 1.f : 0.f;
}

// Likelihood row of step k scaled to a maximum of 1; returns log of the
// maximum (a row with no positive finite maximum is flagged).
template <int K>
KS_DEV void load_raw(const float* __restrict__ src, int64_t k, float (&v)[K]) {
#pragma unroll
    for (int x = 0; x < K; ++x) v[x] = __ldg(src + k * K + x);
}

template <int K>
KS_DEV float scale_lik(float (&l)[K], Flags& bad) {
    float m = 0.f;
#pragma unroll
    for (int x = 0; x < K; ++x) m = fmaxf(m, l[x]);
    bad |= !(m > 0.f) || !(m <= 3.0e38f);
    const float r = 1.f / m;
#pragma unroll
    for (int x = 0; x < K; ++x) l[x] *= r;
    return __logf(m);
}

template <int K>
KS_DEV float load_lik(const float* __restrict__ lik, int64_t k, float (&l)[K], Flags& bad) {
    load_raw<K>(lik, k, l);
    return scale_lik<K>(l, bad);
}

// Definition 1, a_i (x) a_j for general elements (i earlier).  With
// w(y) = exp(lg_j(y) - max lg_j):
//   d(z) = sum_y f_i(y | z) w(y),  f_ij(x | z) = sum_y f_i(y | z) w(y) f_j(x | y) / d(z),
//   lg_ij(z) = lg_i(z) + max lg_j + log d(z).
template <int K>
KS_DEV FE<K> fcombine(FE<K> ei, const FE<K>& ej, Flags& bad) {   // ei is overwritten row by row
    float mx = ej.lg[0];
#pragma unroll
    for (int y = 1; y < K; ++y) mx = fmaxf(mx, ej.lg[y]);
    float w[K];
#pragma unroll
    for (int y = 0; y < K; ++y) w[y] = __expf(ej.lg[y] - mx);
#pragma unroll
    for (int z = 0; z < K; ++z) {
        float fw[K], d = 0.f;
#pragma unroll
        for (int y = 0; y < K; ++y) {
            fw[y] = ei.f[z * K + y] * w[y];
            d += fw[y];
        }
        bad |= !(d > 0.f);
        const float rd = 1.f / d;
#pragma unroll
        for (int x = 0; x < K; ++x) {
            float s = 0.f;
#pragma unroll
            for (int y = 0; y < K; ++y) s = fmaf(fw[y], ej.f[y * K + x], s);
            ei.f[z * K + x] = s * rd;
        }
        ei.lg[z] += mx + __logf(d);
    }
    return ei;
}

// Prefix state (identical rows p, constant L) (x) general element.
template <int K>
KS_DEV void fadvance(FS<K>& st, const FE<K>& e, Flags& bad) {
    float mx = e.lg[0];
#pragma unroll
    for (int y = 1; y < K; ++y) mx = fmaxf(mx, e.lg[y]);
    float v[K], d = 0.f;
#pragma unroll
    for (int y = 0; y < K; ++y) {
        v[y] = st.p[y] * __expf(e.lg[y] - mx);
        d += v[y];
    }
    bad |= !(d > 0.f);
    const float rd = 1.f / d;
    float p[K];
#pragma unroll
    for (int x = 0; x < K; ++x) {
        float s = 0.f;
#pragma unroll
        for (int y = 0; y < K; ++y) s = fmaf(v[y], e.f[y * K + x], s);
        p[x] = s * rd;
    }
#pragma unroll
    for (int x = 0; x < K; ++x) st.p[x] = p[x];
    st.L += mx + __logf(d);
}

// Aggregate (x) step element, with l the scaled likelihood row and lm the log
// of its scale (see the header).  Pi is read from shared memory.
template <int K>
KS_DEV void ffold_step(FE<K>& acc, const float* __restrict__ Pi, const float (&l)[K], float lm, Flags& bad) {
    float row[K][K];   // row[z][x] accumulates (f Pi)[z][x], one Pi row at a time
#pragma unroll
    for (int z = 0; z < K; ++z)
#pragma unroll
        for (int x = 0; x < K; ++x) row[z][x] = 0.f;
#pragma unroll
    for (int y = 0; y < K; ++y) {
        float pr[K];
        load_row<K>(Pi, y, pr);
#pragma unroll
        for (int z = 0; z < K; ++z)
#pragma unroll
            for (int x = 0; x < K; ++x) row[z][x] = fmaf(acc.f[z * K + y], pr[x], row[z][x]);
    }
#pragma unroll
    for (int z = 0; z < K; ++z) {
        float r = 0.f;
#pragma unroll
        for (int x = 0; x < K; ++x) {
            row[z][x] *= l[x];
            r += row[z][x];
        }
        bad |= !(r > 0.f);
        const float rr = 1.f / r;
#pragma unroll
        for (int x = 0; x < K; ++x) acc.f[z * K + x] = row[z][x] * rr;
        acc.lg[z] += lm + __logf(r);
    }
}

// The step element itself (fold of the identity).
template <int K>
KS_DEV void step_element(FE<K>& e, const float* __restrict__ Pi, const float (&l)[K], float lm, Flags& bad) {
#pragma unroll
    for (int z = 0; z < K; ++z) {
        float r = 0.f;
#pragma unroll
        for (int x = 0; x < K; ++x) {
            e.f[z * K + x] = Pi[z * K + x] * l[x];
            r += e.f[z * K + x];
        }
        bad |= !(r > 0.f);
        const float rr = 1.f / r;
#pragma unroll
        for (int x = 0; x < K; ++x) e.f[z * K + x] *= rr;
        e.lg[z] = lm + __logf(r);
    }
}

// Step 1's element as a prefix state: p(x_1 | y_1) and log p(y_1).
template <int K>
KS_DEV void first_state(FS<K>& st, const float (&q1)[K], const float (&l)[K], float lm, Flags& bad) {
    float c = 0.f;
#pragma unroll
    for (int x = 0; x < K; ++x) {
        st.p[x] = q1[x] * l[x];
        c += st.p[x];
    }
    bad |= !(c > 0.f);
    const float rc = 1.f / c;
#pragma unroll
    for (int x = 0; x < K; ++x) st.p[x] *= rc;
    st.L = lm + __logf(c);
}

// Prefix state (x) step element: p' = (p Pi) . l / c, L' = L + log c + lm.
template <int K>
KS_DEV void fadvance_step(FS<K>& st, const float* __restrict__ Pi, const float (&l)[K], float lm, float& comp,
                          Flags& bad) {
    float v[K], c = 0.f;
#pragma unroll
    for (int x = 0; x < K; ++x) v[x] = 0.f;
#pragma unroll
    for (int y = 0; y < K; ++y) {
        float pr[K];
        load_row<K>(Pi, y, pr);
#pragma unroll
        for (int x = 0; x < K; ++x) v[x] = fmaf(st.p[y], pr[x], v[x]);
    }
#pragma unroll
    for (int x = 0; x < K; ++x) {
        v[x] *= l[x];
        c += v[x];
    }
    bad |= !(c > 0.f);
    const float rc = 1.f / c;
#pragma unroll
    for (int x = 0; x < K; ++x) st.p[x] = v[x] * rc;
    // Kahan-compensated running log-likelihood
    const float t = (lm + __logf(c)) - comp;
    const float L = st.L + t;
    comp = (L - st.L) - t;
    st.L = L;
}

// Smoothing element of step k from its filtered marginal p (k < n):
// a(x | z) = p(x) Pi[x][z] / sum_x' p(x') Pi[x'][z].
template <int K>
KS_DEV void selem(SE<K>& e, const float* __restrict__ PiT, const float (&p)[K], Flags& bad) {
#pragma unroll
    for (int z = 0; z < K; ++z) {
        float pc[K], d = 0.f;
        load_row<K>(PiT, z, pc);   // column z of Pi
#pragma unroll
        for (int x = 0; x < K; ++x) {
            e.a[z * K + x] = p[x] * pc[x];
            d += e.a[z * K + x];
        }
        bad |= !(d > 0.f);
        const float rd = 1.f / d;
#pragma unroll
        for (int x = 0; x < K; ++x) e.a[z * K + x] *= rd;
    }
}

// Smoothing element of the last step: a(x | z) = p_n(x) for every z.
template <int K>
KS_DEV void selem_last(SE<K>& e, const float (&p)[K]) {
#pragma unroll
    for (int z = 0; z < K; ++z)
#pragma unroll
        for (int x = 0; x < K; ++x) e.a[z * K + x] = p[x];
}

// Definition 2 in matrix form: (a_i (x) a_j)[z][x] = sum_y a_j[z][y] a_i[y][x]
// (i earlier), i.e. the product a_j a_i.
// The rows of a product of row-stochastic matrices sum to one in exact
// arithmetic; each row is rescaled to that sum, so that the rounding of the
// total probability does not build up along the look-back's chain of tile
// prefixes (one product per tile).
template <int K>
KS_DEV SE<K> smatmul(SE<K> l, const SE<K>& r) {   // l r, l overwritten row by row
#pragma unroll
    for (int z = 0; z < K; ++z) {
        float o[K], t = 0.f;
#pragma unroll
        for (int x = 0; x < K; ++x) {
            float s = 0.f;
#pragma unroll
            for (int y = 0; y < K; ++y) s = fmaf(l.a[z * K + y], r.a[y * K + x], s);
            o[x] = s;
            t += s;
        }
        const float rt = 1.f / t;
#pragma unroll
        for (int x = 0; x < K; ++x) l.a[z * K + x] = o[x] * rt;
    }
    return l;
}

template <int K>
struct FilterOp {
    using Elem = FE<K>;
    using State = FS<K>;
    KS_DEV static Elem combine(const Elem& a, const Elem& b, Flags& bad) { return fcombine<K>(a, b, bad); }
    KS_DEV static void advance(State& s, const Elem& e, Flags& bad) { fadvance<K>(s, e, bad); }
    KS_DEV static void identity(Elem& e) { set_identity<K>(e); }
    KS_DEV static void zero_state(State& s) {
#pragma unroll
        for (int x = 0; x < K; ++x) s.p[x] = 0.f;
        s.L = 0.f;
    }
    KS_DEV static State state_of(const Elem& e) {   // identical rows
        State s;
#pragma unroll
        for (int x = 0; x < K; ++x) s.p[x] = e.f[x];
        s.L = e.lg[0];
        return s;
    }
};

// Reverse scan in scan (reversed-time) order: x (x)_r y = y (x) x, which in
// matrix form is x.a y.a.
template <int K>
struct SmootherOp {
    using Elem = SE<K>;
    using State = SS<K>;
    KS_DEV static Elem combine(const Elem& a, const Elem& b, Flags&) { return smatmul<K>(a, b); }
    KS_DEV static void advance(State& s, const Elem& e, Flags&) {   // s <- s e.a, rescaled to sum 1
        float o[K], t = 0.f;
#pragma unroll
        for (int x = 0; x < K; ++x) {
            float v = 0.f;
#pragma unroll
            for (int z = 0; z < K; ++z) v = fmaf(s.s[z], e.a[z * K + x], v);
            o[x] = v;
            t += v;
        }
        const float rt = 1.f / t;
#pragma unroll
        for (int x = 0; x < K; ++x) s.s[x] = o[x] * rt;
    }
    KS_DEV static void identity(Elem& e) { set_identity<K>(e); }
    KS_DEV static void zero_state(State& s) {
#pragma unroll
        for (int x = 0; x < K; ++x) s.s[x] = 0.f;
    }
    KS_DEV static State state_of(const Elem& e) {
        State s;
#pragma unroll
        for (int x = 0; x < K; ++x) s.s[x] = e.a[x];
        return s;
    }
};

// ---------------------------------------------------------------- kernels
// Model constants (q1 = pi Pi) and the scans' counters and flags.
template <int K>
__global__ void __launch_bounds__(64) hmm_prep_kernel(const float* __restrict__ pi, const float* __restrict__ Pi,
                                                      Const<K>* __restrict__ out, uint32_t* __restrict__ status,
                                                      uint32_t* __restrict__ zero, int nzero) {
    const int t = threadIdx.x;
    for (int i = t; i < nzero; i += blockDim.x) zero[i] = 0u;
    Flags bad = 0u;
    for (int e = t; e < K * K; e += blockDim.x) {
        const float v = Pi[e];
        bad |= !(v >= 0.f) || !(v <= 3.0e38f);
        out->Pi[e] = v;
        out->PiT[(e % K) * K + e / K] = v;
    }
    for (int e = t; e < (4 - K % 4) % 4; e += blockDim.x) out->pad[e] = 0.f;
    for (int x = t; x < K; x += blockDim.x) {
        float s = 0.f;
        for (int y = 0; y < K; ++y) s = fmaf(pi[y], Pi[y * K + x], s);
        bad |= !(s >= 0.f) || !(s <= 3.0e38f);
        out->q1[x] = s;
    }
    report_flags(status, bad, kFull, (t & 31) == 0);
}

template <int K>
KS_DEV void load_const(const Const<K>* __restrict__ g, Const<K>& s, int tid, int nt) {
    const float* src = reinterpret_cast<const float*>(g);
    float* dst = reinterpret_cast<float*>(&s);
    for (int i = tid; i < (int)(sizeof(Const<K>) / 4); i += nt) dst[i] = __ldg(src + i);
}

// Forward scan: filtered marginals filt [T][K], running log-likelihoods
// loglik [T] (may be null), and each thread's smoothing aggregate (its CH
// steps' Definition 2 elements folded forward) in sagg.
template <int K, int NT, int CH>
__global__ void __launch_bounds__(NT) hmm_filter_kernel(const Const<K>* __restrict__ cg,
                                                        const float* __restrict__ lik, int64_t T,
                                                        float* __restrict__ filt, float* __restrict__ loglik,
                                                        ScanState ss, float* __restrict__ sagg) {
    using BS = BlockScan<FilterOp<K>, NT>;
    constexpr int64_t TILE = (int64_t)NT * CH;
    __shared__ __align__(16) Const<K> mc;
    __shared__ typename BS::Smem bsm;
    __shared__ int s_tile;
    const int tid = threadIdx.x;
    load_const<K>(cg, mc, tid, NT);
    if (tid == 0) s_tile = (int)atomicAdd(ss.counter, 1u);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= (int)gridDim.x) return;   // a tile number past the grid (only when the counter was offset)
    const int64_t k0 = tile * TILE + (int64_t)tid * CH;
    const bool valid = k0 < T;
    Flags bad = 0u;

    // ---- phase 1: fold this thread's steps
    FE<K> acc;
    if (!valid) {
        set_identity<K>(acc);
    } else {
        float l[K];
        const float lm = load_lik<K>(lik, k0, l, bad);
        if (k0 == 0) {        // step 1: rows p(x_1 | y_1), g = p(y_1)
            FS<K> s1;
            first_state<K>(s1, mc.q1, l, lm, bad);
#pragma unroll
            for (int z = 0; z < K; ++z) {
#pragma unroll
                for (int x = 0; x < K; ++x) acc.f[z * K + x] = s1.p[x];
                acc.lg[z] = s1.L;
            }
        } else {
            step_element<K>(acc, mc.Pi, l, lm, bad);
        }
        // the next step's likelihood row is loaded while the current one folds
        float ln[K];
        const int last = (int)((k0 + CH <= T ? k0 + CH : T) - k0);
        if (1 < last) load_raw<K>(lik, k0 + 1, ln);
#pragma unroll 1
        for (int i = 1; i < last; ++i) {
#pragma unroll
            for (int x = 0; x < K; ++x) l[x] = ln[x];
            if (i + 1 < last) load_raw<K>(lik, k0 + i + 1, ln);
            const float lmk = scale_lik<K>(l, bad);
            ffold_step<K>(acc, mc.Pi, l, lmk, bad);
        }
    }

    // ---- phase 2
    FS<K> st;
    bool has = false;
    BS::run(bsm, ss, tile, acc, st, has, bad);

    // ---- phase 3: step through the block from the incoming prefix
    if (valid) {
        SE<K> sacc;
        float comp = 0.f, probe = 0.f;
        const int last = (int)((k0 + CH <= T ? k0 + CH : T) - k0);
        float ln[K];
        load_raw<K>(lik, k0, ln);
#pragma unroll 1
        for (int i = 0; i < last; ++i) {
            const int64_t k = k0 + i;
            float l[K];
#pragma unroll
            for (int x = 0; x < K; ++x) l[x] = ln[x];
            if (i + 1 < last) load_raw<K>(lik, k + 1, ln);
            const float lm = scale_lik<K>(l, bad);
            if (!has) {   // only step 1
                first_state<K>(st, mc.q1, l, lm, bad);
                has = true;
            } else {
                fadvance_step<K>(st, mc.Pi, l, lm, comp, bad);
            }
#pragma unroll
            for (int x = 0; x < K; ++x) {
                filt[k * K + x] = st.p[x];
                probe += st.p[x];
            }
            if (loglik) loglik[k] = st.L;
            probe += st.L;
            SE<K> e;
            if (k == T - 1) selem_last<K>(e, st.p);
            else selem<K>(e, mc.PiT, st.p, bad);
            sacc = (i == 0) ? e : smatmul<K>(e, sacc);   // a_k0 (x) ... (x) a_k = a_k ... a_k0
        }
        store_plain(sagg + (k0 / CH) * (int64_t)(sizeof(SE<K>) / 4), sacc);
        bad |= !isfinite(probe);
    }
    report_flags(ss.status, bad, kFull, (tid & 31) == 0);
}

// Reverse scan over the forward scan's per-thread smoothing aggregates; each
// thread then walks its steps backwards from the suffix after them, writing
// smooth [T][K].
template <int K, int NT, int CH>
__global__ void __launch_bounds__(NT) hmm_smoother_kernel(const Const<K>* __restrict__ cg,
                                                          const float* __restrict__ filt, int64_t T,
                                                          float* __restrict__ smooth, ScanState ss,
                                                          const float* __restrict__ sagg) {
    using BS = BlockScan<SmootherOp<K>, NT>;
    __shared__ __align__(16) Const<K> mc;
    __shared__ typename BS::Smem bsm;
    __shared__ int s_tile;
    const int tid = threadIdx.x;
    load_const<K>(cg, mc, tid, NT);
    if (tid == 0) s_tile = (int)atomicAdd(ss.counter, 1u);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= (int)gridDim.x) return;   // a tile number past the grid (only when the counter was offset)
    const int64_t nblk = (T + CH - 1) / CH;
    const int64_t c = nblk - 1 - ((int64_t)tile * NT + tid);   // forward block index
    const bool valid = c >= 0;
    const int64_t klo = c * CH;
    const int64_t khi = valid ? ((klo + CH < T ? klo + CH : T) - 1) : -1;
    Flags bad = 0u;

    SE<K> acc;
    if (valid) acc = load_cg<SE<K>>(sagg + c * (int64_t)(sizeof(SE<K>) / 4));
    else set_identity<K>(acc);

    SS<K> st;
    bool has = false;
    BS::run(bsm, ss, tile, acc, st, has, bad);

    if (valid) {
        float probe = 0.f;
        float pn[K];
        load_raw<K>(filt, khi, pn);
#pragma unroll 1
        for (int64_t k = khi; k >= klo; --k) {
            float p[K];
#pragma unroll
            for (int x = 0; x < K; ++x) p[x] = pn[x];
            if (k > klo) load_raw<K>(filt, k - 1, pn);
            SE<K> e;
            if (k == T - 1) selem_last<K>(e, p);
            else selem<K>(e, mc.PiT, p, bad);
            if (!has) { st = SmootherOp<K>::state_of(e); has = true; }   // only k = T - 1
            else SmootherOp<K>::advance(st, e, bad);
#pragma unroll
            for (int x = 0; x < K; ++x) {
                smooth[k * K + x] = st.s[x];
                probe += st.s[x];
            }
        }
        bad |= !isfinite(probe);
    }
    report_flags(ss.status, bad, kFull, (tid & 31) == 0);
}

}  // namespace hmm
}  // namespace ks
