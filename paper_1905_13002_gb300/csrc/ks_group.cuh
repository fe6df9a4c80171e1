// ks_group.cuh -- elements of larger state size (nx >= 8), one warp per chain.
//
// An element's matrices live in a per-chain shared-memory slot, row-major with
// a padded row pitch; one group of lanes serves one chain and lane r of the
// group computes row r of every result (rows r >= N are idle), reading the
// other operand's rows from shared memory (the group reads one address:
// broadcast).  A group is 8 lanes for N <= 8 (four chains per warp) and the
// whole warp otherwise; groups synchronise and exchange values with masks
// of their own lanes only.  Registers hold a few rows.
// The operators are the same Lemmas 3-6 as the register version in
// ks_ops.cuh; symmetric results are symmetrised as (X + X^T) / 2.
#pragma once

#include "ks_ops.cuh"

namespace ks {
namespace grp {

constexpr unsigned kFullMask = 0xffffffffu;

template <int N>
struct Dim {
    // Row pitch (floats), odd: lane r reading its own row (address r NP + k)
    // then hits bank (r + k) mod 32, distinct across the warp; broadcast reads
    // (one address) and column reads (lane r reads column r) are conflict free
    // at any pitch.  It also holds the 2 ny scalars per row of the rank-ny
    // products (ny <= nx / 2 here).
    static constexpr int NP = N + 1;
    static constexpr int MAT = N * NP;          // one matrix
    static constexpr int FSLOT = 3 * MAT + 2 * NP;   // A, C, J, b, eta
    static constexpr int SSLOT = 2 * MAT + NP;       // E, L, g
};

// Filtering element slot: A, C, J (N x NP each), b, eta (NP each).
template <int N>
struct FSlot {
    float* p;
    KS_DEV float* A() const { return p; }
    KS_DEV float* C() const { return p + Dim<N>::MAT; }
    KS_DEV float* J() const { return p + 2 * Dim<N>::MAT; }
    KS_DEV float* b() const { return p + 3 * Dim<N>::MAT; }
    KS_DEV float* eta() const { return p + 3 * Dim<N>::MAT + Dim<N>::NP; }
};

// Smoothing element slot: E, L (N x NP), g (NP).
template <int N>
struct SSlot {
    float* p;
    KS_DEV float* E() const { return p; }
    KS_DEV float* L() const { return p + Dim<N>::MAT; }
    KS_DEV float* g() const { return p + 2 * Dim<N>::MAT; }
};

// Lanes per chain and the mask of the calling lane's group.
template <int N>
struct Grp {
    static constexpr int GS = N <= 8 ? 8 : 32;
};
template <int N>
KS_DEV unsigned gmask() {
    if constexpr (Grp<N>::GS == 32) {
        return kFullMask;
    } else {
        constexpr unsigned ones = (1u << Grp<N>::GS) - 1u;
        return ones << ((threadIdx.x & 31) & ~(Grp<N>::GS - 1));
    }
}
template <int N>
KS_DEV void gsync() { __syncwarp(gmask<N>()); }

// ---------------------------------------------------------------- row kernels
// Left operands are rows in shared memory (pointers), so that for large N the
// inner-product loop can stay rolled without indexing a register array; the
// output row is a register array with a compile-time index.
template <int N>
struct Unroll {
    static constexpr int K = N <= 16 ? N : 4;
};

template <int N>
KS_DEV void load_row(const float* X, int r, float (&x)[N]) {
    const float* p = X + r * Dim<N>::NP;
#pragma unroll
    for (int c = 0; c < N; ++c) x[c] = p[c];
}
template <int N>
KS_DEV void store_row(float* X, int r, const float (&x)[N]) {
    float* p = X + r * Dim<N>::NP;
#pragma unroll
    for (int c = 0; c < N; ++c) p[c] = x[c];
}
// x = y Z       (x[c] = sum_k y[k] Z[k][c]); y: a row in shared memory
template <int N>
KS_DEV void row_mul(const float* y, const float* Z, float (&x)[N]) {
#pragma unroll
    for (int c = 0; c < N; ++c) x[c] = 0.f;
#pragma unroll Unroll<N>::K
    for (int k = 0; k < N; ++k) {
        const float yk = y[k];
        const float* zr = Z + k * Dim<N>::NP;
#pragma unroll
        for (int c = 0; c < N; ++c) x[c] = fmaf(yk, zr[c], x[c]);
    }
}
// x = y Z^T     (x[c] = sum_k y[k] Z[c][k])
template <int N>
KS_DEV void row_mulT(const float* y, const float* Z, float (&x)[N]) {
#pragma unroll
    for (int c = 0; c < N; ++c) x[c] = 0.f;
#pragma unroll Unroll<N>::K
    for (int k = 0; k < N; ++k) {
        const float yk = y[k];
#pragma unroll
        for (int c = 0; c < N; ++c) x[c] = fmaf(yk, Z[c * Dim<N>::NP + k], x[c]);
    }
}
// x = (Y^T Z)[r] (x[c] = sum_k Y[k][r] Z[k][c])
template <int N>
KS_DEV void colT_mul(const float* Y, int r, const float* Z, float (&x)[N]) {
#pragma unroll
    for (int c = 0; c < N; ++c) x[c] = 0.f;
#pragma unroll Unroll<N>::K
    for (int k = 0; k < N; ++k) {
        const float yk = Y[k * Dim<N>::NP + r];
        const float* zr = Z + k * Dim<N>::NP;
#pragma unroll
        for (int c = 0; c < N; ++c) x[c] = fmaf(yk, zr[c], x[c]);
    }
}
// x = y C_const, C_const an N x N row-major (pitch N) constant matrix
template <int N>
KS_DEV void row_mul_const(const float* y, const float* Cc, float (&x)[N]) {
#pragma unroll
    for (int c = 0; c < N; ++c) x[c] = 0.f;
#pragma unroll Unroll<N>::K
    for (int k = 0; k < N; ++k) {
        const float yk = y[k];
#pragma unroll
        for (int c = 0; c < N; ++c) x[c] = fmaf(yk, Cc[k * N + c], x[c]);
    }
}
// x = y Cc^T (x[c] = sum_k y[k] Cc[c][k]), Cc pitch N
template <int N>
KS_DEV void row_mulT_const(const float* y, const float* Cc, float (&x)[N]) {
#pragma unroll
    for (int c = 0; c < N; ++c) x[c] = 0.f;
#pragma unroll Unroll<N>::K
    for (int k = 0; k < N; ++k) {
        const float yk = y[k];
#pragma unroll
        for (int c = 0; c < N; ++c) x[c] = fmaf(yk, Cc[c * N + k], x[c]);
    }
}
template <int N>
KS_DEV float dot(const float* y, const float* v) {
    float s = 0.f;
#pragma unroll Unroll<N>::K
    for (int k = 0; k < N; ++k) s = fmaf(y[k], v[k], s);
    return s;
}
// sum_k Y[k][r] v[k]
template <int N>
KS_DEV float col_dot(const float* Y, int r, const float* v) {
    float s = 0.f;
#pragma unroll Unroll<N>::K
    for (int k = 0; k < N; ++k) s = fmaf(Y[k * Dim<N>::NP + r], v[k], s);
    return s;
}
template <int N>
KS_DEV const float* rowp(const float* X, int r) { return X + r * Dim<N>::NP; }
// x = y Z with y any row pointer (e.g. a constant matrix row) and Z rows of pitch NP
template <int N>
KS_DEV void row_mul_const_rows(const float* y, const float* Z, float (&x)[N]) { row_mul<N>(y, Z, x); }

// ---------------------------------------------------------------- Gauss-Jordan
// Inverse of the N x N matrix whose row r is `m` (lane r), with partial
// pivoting; the pivot row is chosen by a warp-wide argmax of |column k| over
// the rows not yet used and broadcast through `pr` (2 NP floats of shared
// memory).  Rows are not exchanged: after the elimination, row r of the
// inverse sits on the lane that pivoted column r, and is moved to lane r
// through `out` (an N x NP matrix), where the result ends (row r on lane r).
template <int N>
KS_DEV bool gj_inverse(int r, float (&m)[N], float* pr, float* out) {
    const bool act = r < N;
    float inv[N];
#pragma unroll
    for (int c = 0; c < N; ++c) inv[c] = (act && c == r) ? 1.f : 0.f;
    bool used = !act;
    bool ok = true;
    int src = 0;   // lane holding row r of the inverse
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
        float v = -1.f;
#pragma unroll
        for (int c = 0; c < N; ++c)
            if (c == k) v = used ? -1.f : fabsf(m[c]);
        int idx = r;
#pragma unroll
        for (int off = Grp<N>::GS / 2; off > 0; off >>= 1) {
            const float ov = __shfl_xor_sync(gmask<N>(), v, off);
            const int oi = __shfl_xor_sync(gmask<N>(), idx, off);
            if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
        }
        const int p = idx;
        if (r == p) {
            used = true;
#pragma unroll
            for (int c = 0; c < N; ++c) { pr[c] = m[c]; pr[Dim<N>::NP + c] = inv[c]; }
        }
        if (r == k) src = p;
        gsync<N>();
        float piv = 0.f;
#pragma unroll
        for (int c = 0; c < N; ++c)
            if (c == k) piv = pr[c];
        ok = ok && isfinite(piv) && fabsf(piv) > 1e-30f;
        const float ip = __frcp_rn(piv);
        if (r == p) {
#pragma unroll
            for (int c = 0; c < N; ++c) { m[c] = pr[c] * ip; inv[c] = pr[Dim<N>::NP + c] * ip; }
        } else if (act) {
            float f = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c)
                if (c == k) f = m[c];
            const float fi = f * ip;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                m[c] = fmaf(-fi, pr[c], m[c]);
                inv[c] = fmaf(-fi, pr[Dim<N>::NP + c], inv[c]);
            }
        }
        gsync<N>();
    }
    if (act) store_row<N>(out, r, inv);
    gsync<N>();
    float res[N];
    load_row<N>(out, act ? src : 0, res);
    gsync<N>();
    if (act) store_row<N>(out, r, res);
    gsync<N>();
    return ok;
}

// Maximum of v over the lane group.
template <int N>
KS_DEV float gmax(float v) {
#pragma unroll
    for (int off = Grp<N>::GS / 2; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(gmask<N>(), v, off));
    return v;
}

// Lemma 4's M^{-1} for M = I + C J, from row r of M on lane r (`m`,
// destroyed): gj_inverse (rows of the result in `out`), then, when the
// infinity-norm condition estimate ||M||_inf ||M^{-1}||_inf exceeds
// kRefineCond, one refinement step: lane r forms row r of M and of the
// residual R = I - M X in FP64 from the FP32 rows of C and J (full, pitch NP)
// and all rows of X = out, parks R in the scratch matrix `Rs`, and replaces
// its row of X by the row of X + X R.  Returns FL_BAD on a failed pivot,
// FL_REFINED when the refinement ran, else 0.
template <int N>
KS_DEV Flags ginverse_cj(int r, float (&m)[N], const float* C, const float* J, float* pr, float* out,
                         float* Rs) {
    constexpr int NP = Dim<N>::NP;
    const bool act = r < N;
    float rs = 0.f;
#pragma unroll
    for (int c = 0; c < N; ++c) rs += fabsf(m[c]);
    const float nm = gmax<N>(act ? rs : 0.f);
    if (!gj_inverse<N>(r, m, pr, out)) return FL_BAD;
    float xs = 0.f;
    if (act) {
#pragma unroll
        for (int c = 0; c < N; ++c) xs += fabsf(out[r * NP + c]);
    }
    const float cond = nm * gmax<N>(xs);
    if (!(cond > kRefineCond) || !(cond < 3.0e38f)) return 0u;   // uniform over the group
    if (act) {
        double md[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double t = (c == r) ? 1.0 : 0.0;
#pragma unroll Unroll<N>::K
            for (int k = 0; k < N; ++k) t = fma((double)C[r * NP + k], (double)J[k * NP + c], t);
            md[c] = t;
        }
        float rr[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double t = (c == r) ? 1.0 : 0.0;
#pragma unroll Unroll<N>::K
            for (int k = 0; k < N; ++k) t = fma(-md[k], (double)out[k * NP + c], t);
            rr[c] = (float)t;
        }
        store_row<N>(Rs, r, rr);
    }
    gsync<N>();
    if (act) {
        float xn[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
            float t = out[r * NP + c];
#pragma unroll Unroll<N>::K
            for (int k = 0; k < N; ++k) t = fmaf(out[r * NP + k], Rs[k * NP + c], t);
            xn[c] = t;
        }
        store_row<N>(out, r, xn);   // other lanes read only their own row of out here
    }
    gsync<N>();
    return FL_REFINED;
}

// (X + X^T)/2 of a matrix with rows in `tmp`, written row r to `dst`.
template <int N>
KS_DEV void symmetrise_into(int r, const float* tmp, float* dst) {
    if (r < N) {
        float x[N];
#pragma unroll
        for (int c = 0; c < N; ++c) x[c] = 0.5f * (tmp[r * Dim<N>::NP + c] + tmp[c * Dim<N>::NP + r]);
        store_row<N>(dst, r, x);
    }
}

// Scratch of one warp: six N x NP matrices and eight NP vectors.
template <int N>
struct Scratch {
    float* p;
    KS_DEV float* S(int i) const { return p + i * Dim<N>::MAT; }
    KS_DEV float* V(int i) const { return p + 6 * Dim<N>::MAT + i * Dim<N>::NP; }
    static constexpr int FLOATS = 6 * Dim<N>::MAT + 8 * Dim<N>::NP;
};

// ---------------------------------------------------------------- Lemma 4
// o = i (x) j (general filtering operator), o distinct from i and j.
//   M = I + C_i J_j, Mi = M^{-1};  A_o = A_j Mi A_i,
//   b_o = A_j Mi (b_i + C_i eta_j) + b_j,   C_o = A_j Mi C_i A_j^T + C_j,
//   eta_o = A_i^T Mi^T (eta_j - J_j b_i) + eta_i,   J_o = A_i^T (Mi^T J_j) A_i + J_i.
// Scratch: S0 Mi, S1 T1 = (Mi^T J_j) A_i, S2 X C_i then C_o, S3 J_o, S4 X = A_j Mi,
// S5 Mi^T J_j;  V0 t, V1 v, V2 Mi^T v, V6-V7 pivots.
template <int N>
KS_DEV void fcombine(int r, FSlot<N> i, FSlot<N> j, FSlot<N> o, Scratch<N> s, Flags& bad) {
    const bool act = r < N;
    const int rr = act ? r : 0;
    float m[N];
    row_mul<N>(rowp<N>(i.C(), rr), j.J(), m);
#pragma unroll
    for (int c = 0; c < N; ++c) m[c] += (act && c == r) ? 1.f : 0.f;
    if (act) {
        s.V(0)[r] = i.b()[r] + dot<N>(rowp<N>(i.C(), r), j.eta());   // t = b_i + C_i eta_j
        s.V(1)[r] = j.eta()[r] - dot<N>(rowp<N>(j.J(), r), i.b());   // v = eta_j - J_j b_i
    }
    bad |= ginverse_cj<N>(r, m, i.C(), j.J(), s.V(6), s.S(0), s.S(4));   // Mi rows in S0
    {
        float x[N], v[N];
        row_mul<N>(rowp<N>(j.A(), rr), s.S(0), x);                   // X = A_j Mi
        colT_mul<N>(s.S(0), rr, j.J(), v);                           // Mi^T J_j
        if (act) {
            store_row<N>(s.S(4), r, x);
            store_row<N>(s.S(5), r, v);
            s.V(2)[r] = col_dot<N>(s.S(0), r, s.V(1));               // w = Mi^T v
        }
    }
    gsync<N>();
    {
        float t1[N], wc[N], an[N];
        row_mul<N>(rowp<N>(s.S(5), rr), i.A(), t1);                  // T1 = (Mi^T J_j) A_i
        row_mul<N>(rowp<N>(s.S(4), rr), i.C(), wc);                  // X C_i
        row_mul<N>(rowp<N>(s.S(4), rr), i.A(), an);                  // A_o = X A_i
        if (act) {
            store_row<N>(s.S(1), r, t1);
            store_row<N>(s.S(2), r, wc);
            store_row<N>(o.A(), r, an);
            o.b()[r] = dot<N>(rowp<N>(s.S(4), r), s.V(0)) + j.b()[r];
            o.eta()[r] = col_dot<N>(i.A(), r, s.V(2)) + i.eta()[r];
        }
    }
    gsync<N>();
    {
        float cr[N], jn[N];
        row_mulT<N>(rowp<N>(s.S(2), rr), j.A(), cr);                 // (X C_i) A_j^T
        colT_mul<N>(i.A(), rr, s.S(1), jn);                          // A_i^T T1
        if (act) {
#pragma unroll
            for (int c = 0; c < N; ++c) {
                cr[c] += j.C()[r * Dim<N>::NP + c];
                jn[c] += i.J()[r * Dim<N>::NP + c];
            }
        }
        gsync<N>();                                                     // S2 row r (X C_i) is read by lane r only
        if (act) {
            store_row<N>(s.S(2), r, cr);
            store_row<N>(s.S(3), r, jn);
        }
    }
    gsync<N>();
    symmetrise_into<N>(r, s.S(2), o.C());
    symmetrise_into<N>(r, s.S(3), o.J());
    gsync<N>();
}

// o = (b, C) (x) j for a prefix state (A = 0); only b and C of o are formed:
//   b_o = A_j Mi (b + C eta_j) + b_j,  C_o = A_j Mi C A_j^T + C_j.
template <int N>
KS_DEV void fadvance(int r, FSlot<N> st, FSlot<N> j, FSlot<N> o, Scratch<N> s, Flags& bad) {
    const bool act = r < N;
    const int rr = act ? r : 0;
    float m[N];
    row_mul<N>(rowp<N>(st.C(), rr), j.J(), m);
#pragma unroll
    for (int c = 0; c < N; ++c) m[c] += (act && c == r) ? 1.f : 0.f;
    if (act) s.V(0)[r] = st.b()[r] + dot<N>(rowp<N>(st.C(), r), j.eta());
    bad |= ginverse_cj<N>(r, m, st.C(), j.J(), s.V(6), s.S(0), s.S(4));
    {
        float x[N];
        row_mul<N>(rowp<N>(j.A(), rr), s.S(0), x);
        if (act) store_row<N>(s.S(4), r, x);
    }
    gsync<N>();
    {
        float wc[N];
        row_mul<N>(rowp<N>(s.S(4), rr), st.C(), wc);
        if (act) store_row<N>(s.S(2), r, wc);
    }
    gsync<N>();
    {
        float cr[N];
        row_mulT<N>(rowp<N>(s.S(2), rr), j.A(), cr);
        if (act) {
#pragma unroll
            for (int c = 0; c < N; ++c) cr[c] += j.C()[r * Dim<N>::NP + c];
            o.b()[r] = dot<N>(rowp<N>(s.S(4), r), s.V(0)) + j.b()[r];
        }
        gsync<N>();
        if (act) store_row<N>(s.S(3), r, cr);
    }
    gsync<N>();
    symmetrise_into<N>(r, s.S(3), o.C());
    gsync<N>();
}

// Rank-M form for a single measurement element j (constants in `mc`):
// J_j = U^T U, eta_j = U^T w.  With G = I + U C_i U^T = L L^T:
//   M^{-1} = I - CUL UL (CUL = C_i U^T L^{-T}, UL = L^{-1} U),
//   X = A M^{-1},  A_o = X A_i,  b_o = X (b_i + C_i U^T w) + b_j,
//   C_o = A (C_i - CUL CUL^T) A^T + C,
//   eta_o = (UL A_i)^T L^{-1} (w - U b_i) + eta_i,  J_o = (UL A_i)^T (UL A_i) + J_i.
// PREFIX: i is a prefix (A_i = 0): only b and C of o are formed.
// Scratch: S0 CU then C_o, S1 [CUL | UL^T], S2 W, S3 VA^T, S4 X, S5 Y;  V0 b_i, V1 t.
template <int N, int M, bool PREFIX>
KS_DEV void fcombine_meas(int r, FSlot<N> i, const ModelConst<N, M>& mc, float bj, const float (&w)[M],
                          FSlot<N> o, Scratch<N> s, Flags& bad) {
    constexpr int NP = Dim<N>::NP;
    const bool act = r < N;
    const int rr = act ? r : 0;
    const float* ci = rowp<N>(i.C(), rr);
    float cu[M];                                             // CU[r][q] = C_i[r] . U[q]
#pragma unroll
    for (int q = 0; q < M; ++q) cu[q] = dot<N>(ci, mc.U + q * N);
    if (act) {
#pragma unroll
        for (int q = 0; q < M; ++q) s.S(0)[r * NP + q] = cu[q];
        s.V(0)[r] = i.b()[r];
    }
    gsync<N>();
    float G[sym_size(M)];                                    // G = I + U CU (every lane)
#pragma unroll
    for (int q = 0; q < M; ++q)
#pragma unroll
        for (int p = 0; p <= q; ++p) {
            float t = (p == q) ? 1.f : 0.f;
#pragma unroll Unroll<N>::K
            for (int a = 0; a < N; ++a) t = fmaf(mc.U[q * N + a], s.S(0)[a * NP + p], t);
            G[sidx(q, p)] = t;
        }
    float Li[M][M];
    bad |= !chol_inv_lower<M>(G, Li);
    float cul[M], ulr[M];
#pragma unroll
    for (int q = 0; q < M; ++q) {
        float t = 0.f, u = 0.f;
#pragma unroll
        for (int p = 0; p <= q; ++p) {
            t = fmaf(cu[p], Li[q][p], t);
            u = fmaf(Li[q][p], mc.U[p * N + rr], u);
        }
        cul[q] = t;                                          // CUL[r][q]
        ulr[q] = u;                                          // UL[q][r]
    }
    float t_r = act ? i.b()[r] : 0.f;
#pragma unroll
    for (int q = 0; q < M; ++q) t_r = fmaf(cu[q], w[q], t_r);
    if (act) {
#pragma unroll
        for (int q = 0; q < M; ++q) {
            s.S(1)[r * NP + q] = cul[q];
            s.S(1)[r * NP + M + q] = ulr[q];
        }
        s.V(1)[r] = t_r;
    }
    gsync<N>();
    {
        const float* ar = mc.A + rr * N;                     // X[r] = A[r] - (A[r] CUL) UL
        float ac[M];
#pragma unroll
        for (int q = 0; q < M; ++q) {
            float t = 0.f;
#pragma unroll Unroll<N>::K
            for (int c = 0; c < N; ++c) t = fmaf(ar[c], s.S(1)[c * NP + q], t);
            ac[q] = t;
        }
        float x[N], wr[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
            float t = ar[c], u = ci[c];
#pragma unroll
            for (int q = 0; q < M; ++q) {
                t = fmaf(-ac[q], s.S(1)[c * NP + M + q], t);
                u = fmaf(-cul[q], s.S(1)[c * NP + q], u);
            }
            x[c] = t;
            wr[c] = u;                                       // W[r] = C_i[r] - CUL[r] CUL^T
        }
        if (act) {
            store_row<N>(s.S(4), r, x);
            store_row<N>(s.S(2), r, wr);
        }
    }
    gsync<N>();
    if (act) o.b()[r] = dot<N>(rowp<N>(s.S(4), r), s.V(1)) + bj;
    if constexpr (!PREFIX) {
        float an[N];
        row_mul<N>(rowp<N>(s.S(4), rr), i.A(), an);          // A_o = X A_i
        float va[M];                                         // VA[q][r] = sum_a UL[q][a] A_i[a][r]
#pragma unroll
        for (int q = 0; q < M; ++q) {
            float t = 0.f;
#pragma unroll Unroll<N>::K
            for (int a = 0; a < N; ++a) t = fmaf(s.S(1)[a * NP + M + q], i.A()[a * NP + rr], t);
            va[q] = t;
        }
        float sv[M];                                         // sv = Li (w - U b_i)
        {
            float rv[M];
#pragma unroll
            for (int q = 0; q < M; ++q) rv[q] = w[q] - dot<N>(mc.U + q * N, s.V(0));
#pragma unroll
            for (int q = 0; q < M; ++q) {
                float t = 0.f;
#pragma unroll
                for (int p = 0; p <= q; ++p) t = fmaf(Li[q][p], rv[p], t);
                sv[q] = t;
            }
        }
        if (act) {
            store_row<N>(o.A(), r, an);
            float e = i.eta()[r];
#pragma unroll
            for (int q = 0; q < M; ++q) {
                e = fmaf(va[q], sv[q], e);
                s.S(3)[r * NP + q] = va[q];
            }
            o.eta()[r] = e;
        }
    }
    {
        float y[N];
        row_mul_const_rows<N>(mc.A + rr * N, s.S(2), y);     // Y[r] = A[r] W
        if (act) store_row<N>(s.S(5), r, y);
    }
    gsync<N>();
    {
        float cr[N];
        row_mulT_const<N>(rowp<N>(s.S(5), rr), mc.A, cr);    // C_o[r] = Y[r] A^T + C[r]
        if (act) {
#pragma unroll
            for (int c = 0; c < N; ++c) cr[c] += mc.C[sidx(r, c)];
            store_row<N>(s.S(0), r, cr);
        }
    }
    if constexpr (!PREFIX) {
        if (act) {
            float jn[N];
#pragma unroll
            for (int c = 0; c < N; ++c) {
                float t = i.J()[r * NP + c];
#pragma unroll
                for (int q = 0; q < M; ++q) t = fmaf(s.S(3)[r * NP + q], s.S(3)[c * NP + q], t);
                jn[c] = t;
            }
            store_row<N>(o.J(), r, jn);                      // VA^T VA + J_i: exactly symmetric
        }
    }
    gsync<N>();
    symmetrise_into<N>(r, s.S(0), o.C());
    gsync<N>();
}

// ---------------------------------------------------------------- Lemma 3 rows
// Measurement element k > 1 of Lemma 3: e = y - H u - d, b = u + K e (row r),
// w = L_S^{-1} e (all lanes).
template <int N, int M>
KS_DEV float meas(int r, const ModelConst<N, M>& mc, const float* __restrict__ yk, float (&w)[M]) {
    float e[M];
#pragma unroll
    for (int q = 0; q < M; ++q) e[q] = __ldg(yk + q) - mc.hud[q];
#pragma unroll
    for (int q = 0; q < M; ++q) {
        float t = 0.f;
#pragma unroll
        for (int p = 0; p <= q; ++p) t = fmaf(mc.Lsi[q * M + p], e[p], t);
        w[q] = t;
    }
    const int rr = r < N ? r : 0;
    float b = mc.u[rr];
#pragma unroll
    for (int q = 0; q < M; ++q) b = fmaf(mc.K[rr * M + q], e[q], b);
    return b;
}

// The measurement element in general form: A, C constant, J = U^T U, eta = U^T w.
template <int N, int M>
KS_DEV void expand_meas(int r, const ModelConst<N, M>& mc, float b, const float (&w)[M], FSlot<N> o) {
    if (r < N) {
        float* pa = o.A() + r * Dim<N>::NP;
        float* pc = o.C() + r * Dim<N>::NP;
        float* pj = o.J() + r * Dim<N>::NP;
#pragma unroll Unroll<N>::K
        for (int q = 0; q < N; ++q) {
            pa[q] = mc.A[r * N + q];
            pc[q] = mc.C[sidx(r, q)];
            float t = 0.f;
#pragma unroll
            for (int p = 0; p < M; ++p) t = fmaf(mc.U[p * N + r], mc.U[p * N + q], t);
            pj[q] = t;
        }
        float e = 0.f;
#pragma unroll
        for (int p = 0; p < M; ++p) e = fmaf(mc.U[p * N + r], w[p], e);
        o.eta()[r] = e;
        o.b()[r] = b;
    }
    gsync<N>();
}

// The k = 1 element: A_1 = 0, b_1, C_1 (built in FP64), eta_1 = 0, J_1 = 0.
template <int N, int M>
KS_DEV void first_elem(int r, const ModelConst<N, M>& mc, FSlot<N> o) {
    if (r < N) {
        float* pa = o.A() + r * Dim<N>::NP;
        float* pc = o.C() + r * Dim<N>::NP;
        float* pj = o.J() + r * Dim<N>::NP;
#pragma unroll Unroll<N>::K
        for (int q = 0; q < N; ++q) { pa[q] = 0.f; pc[q] = mc.C1[sidx(r, q)]; pj[q] = 0.f; }
        o.b()[r] = mc.b1[r];
        o.eta()[r] = 0.f;
    }
    gsync<N>();
}

// acc (x) a_1 for a sequence's first element (A_1 = 0, eta_1 = J_1 = 0):
// (0, b_1, C_1, eta_acc, J_acc), in place.
template <int N, int M>
KS_DEV void reset_first(int r, const ModelConst<N, M>& mc, FSlot<N> acc) {
    if (r < N) {
        float* pa = acc.A() + r * Dim<N>::NP;
        float* pc = acc.C() + r * Dim<N>::NP;
#pragma unroll Unroll<N>::K
        for (int q = 0; q < N; ++q) { pa[q] = 0.f; pc[q] = mc.C1[sidx(r, q)]; }
        acc.b()[r] = mc.b1[r];
    }
    gsync<N>();
}

// Posterior state (b, C) = (b_1, C_1) for a sequence's first step.
template <int N, int M>
KS_DEV void first_state(int r, const ModelConst<N, M>& mc, FSlot<N> st) {
    if (r < N) {
        float* pc = st.C() + r * Dim<N>::NP;
#pragma unroll Unroll<N>::K
        for (int q = 0; q < N; ++q) pc[q] = mc.C1[sidx(r, q)];
        st.b()[r] = mc.b1[r];
    }
    gsync<N>();
}

// ---------------------------------------------------------------- Lemma 5 rows
// Smoothing element from the filtered (xbar, P) (P rows in `P`, xbar in `xb`):
// k < n: FP = F P, P- = FP F^T + Q, E = P F^T (P-)^{-1} = FP^T (P-)^{-1},
//        g = xbar - E (F xbar + u), L = P - E (F P);  k = n: (0, xbar, P).
// Scratch: S0 (P-)^{-1}, S1 FP, S2 L, S4 rows of P-;  V0 F xbar + u, V6-V7 pivots.
template <int N, int M>
KS_DEV void selem(int r, const ModelConst<N, M>& mc, const float* P, const float* xb, bool last, SSlot<N> o,
                  Scratch<N> s, Flags& bad) {
    constexpr int NP = Dim<N>::NP;
    const bool act = r < N;
    const int rr = act ? r : 0;
    if (last) {
        if (act) {
#pragma unroll Unroll<N>::K
            for (int q = 0; q < N; ++q) {
                o.E()[r * NP + q] = 0.f;
                o.L()[r * NP + q] = P[r * NP + q];
            }
            o.g()[r] = xb[r];
        }
        gsync<N>();
        return;
    }
    {
        float fp[N];
        row_mul_const_rows<N>(mc.F + rr * N, P, fp);         // FP[r] = F[r] P
        if (act) {
            store_row<N>(s.S(1), r, fp);
            s.V(0)[r] = dot<N>(mc.F + r * N, xb) + mc.u[r];
        }
    }
    gsync<N>();
    float pm[N];
    row_mulT_const<N>(rowp<N>(s.S(1), rr), mc.F, pm);       // P-[r] = FP[r] F^T + Q[r]
    if (act) {
#pragma unroll
        for (int c = 0; c < N; ++c) pm[c] += mc.Q[sidx(r, c)];
    }
    bad |= !gj_inverse<N>(r, pm, s.V(6), s.S(0));            // (P-)^{-1} rows in S0
    {
        float e[N];
        colT_mul<N>(s.S(1), rr, s.S(0), e);                  // E[r] = (FP^T (P-)^{-1})[r]
        if (act) store_row<N>(o.E(), r, e);
    }
    gsync<N>();
    if (act) {
        o.g()[r] = xb[r] - dot<N>(rowp<N>(o.E(), r), s.V(0));
        float l[N];
        row_mul<N>(rowp<N>(o.E(), r), s.S(1), l);            // (E F P)[r]
#pragma unroll
        for (int q = 0; q < N; ++q) l[q] = P[r * NP + q] - l[q];
        store_row<N>(s.S(2), r, l);
    }
    gsync<N>();
    symmetrise_into<N>(r, s.S(2), o.L());
    gsync<N>();
}

// ---------------------------------------------------------------- Lemma 6 rows
// o = i (x) j, i the earlier step: E = E_i E_j, g = E_i g_j + g_i, L = E_i L_j E_i^T + L_i.
// STATE: j is a suffix (E_j = 0); only g and L are formed.  Scratch: S3, S5.
template <int N, bool STATE>
KS_DEV void scombine(int r, SSlot<N> i, SSlot<N> j, SSlot<N> o, Scratch<N> s) {
    const bool act = r < N;
    const int rr = act ? r : 0;
    {
        float y[N];
        row_mul<N>(rowp<N>(i.E(), rr), j.L(), y);            // Y[r] = E_i[r] L_j
        if (act) store_row<N>(s.S(5), r, y);
    }
    gsync<N>();
    {
        float l[N];
        row_mulT<N>(rowp<N>(s.S(5), rr), i.E(), l);          // L[r][c] = Y[r] . E_i[c]
        if (act) {
#pragma unroll
            for (int q = 0; q < N; ++q) l[q] += i.L()[r * Dim<N>::NP + q];
            store_row<N>(s.S(3), r, l);
            o.g()[r] = dot<N>(rowp<N>(i.E(), r), j.g()) + i.g()[r];
        }
    }
    if constexpr (!STATE) {
        float en[N];
        row_mul<N>(rowp<N>(i.E(), rr), j.E(), en);
        if (act) store_row<N>(o.E(), r, en);
    }
    gsync<N>();
    symmetrise_into<N>(r, s.S(3), o.L());
    gsync<N>();
}

}  // namespace grp
}  // namespace ks
