// ks_ops.cuh -- register-resident elements and operators of Section IV.
//
// Every quantity lives in registers of one thread, with compile-time sizes
// N = nx, M = ny, so all indexing below resolves at compile time.  Symmetric
// matrices (C, J, L, covariances) are kept as their packed lower triangle,
// which makes every symmetric result exactly symmetric (the symmetrisation
// of C, J and L after each combine).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define KS_DEV __device__ __forceinline__

namespace ks {

__host__ __device__ constexpr int sym_size(int n) { return n * (n + 1) / 2; }
__host__ __device__ constexpr int sidx(int i, int j) {
    return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i;
}

// Device status bits (combined with atomicOr into the workspace status word).
enum : uint32_t { ST_NUMERIC = 1u, ST_TIMEOUT = 2u, ST_BADARG = 4u };

// Per-thread diagnostic bits carried through the operators:
//   FL_BAD      a non-finite value or a failed factorisation (reported as ST_NUMERIC);
//   FL_REFINED  an inverse got the FP64-residual refinement step because its
//               condition estimate exceeded kRefineCond;
//   FL_NEED     an inverse's condition estimate exceeded kRefineCond in code
//               that does not refine (the call then repeats the scan with
//               refinement, see the scan kernels).
using Flags = uint32_t;
enum : uint32_t { FL_BAD = 1u, FL_REFINED = 2u, FL_NEED = 4u };

// How the general Lemma 4 operator takes (I + C_i J_j)^{-1}: plain FP32
// Gauss-Jordan; the same with the condition estimate (FL_NEED when it
// exceeds kRefineCond); or with the estimate and the FP64 refinement.
enum : int { REF_NONE = 0, REF_DETECT = 1, REF_FP64 = 2 };

// Condition number (1-norm or infinity-norm estimate) above which an FP32
// inverse gets one refinement step with its residual formed in FP64.
constexpr float kRefineCond = 1.0e3f;

// Workspace header words (the first 256 bytes of every workspace, zeroed by
// ks_workspace_init): [0] status bits, [1] refinement counter, [2] look-back
// wait limit in polls (0: the scan's default), [3] the forward scans' first
// tile number (0; 1 only when a test leaves tile 0 unclaimed to make the
// look-back waits run out), [4] set when a scan without refinement met an
// ill-conditioned inverse (cleared by the preparation kernel).
enum : int { HDR_STATUS = 0, HDR_REFINED = 1, HDR_WAIT = 2, HDR_FIRST_TILE = 3, HDR_NEED = 4 };

// End-of-kernel report of one warp or lane group (`mask`), by its `leader`
// lane: a numeric failure sets ST_NUMERIC in the status word, a group in
// which any lane refined an inverse adds one to the refinement counter, and
// one that met an ill-conditioned inverse without refining it sets HDR_NEED.
KS_DEV void report_flags(uint32_t* status, Flags f, unsigned mask, bool leader) {
    const bool b = __any_sync(mask, (f & FL_BAD) != 0u);
    const bool r = __any_sync(mask, (f & FL_REFINED) != 0u);
    const bool n = __any_sync(mask, (f & FL_NEED) != 0u);
    if (leader && b) atomicOr(status + HDR_STATUS, ST_NUMERIC);
    if (leader && r) atomicAdd(status + HDR_REFINED, 1u);
    if (leader && n) atomicOr(status + HDR_NEED, 1u);
}

// ---------------------------------------------------------------- elements
// Filtering element of Lemma 3: f(x|z) = N(x; A z + b, C), g(z) ∝ N_I(z; eta, J).
template <int N>
struct FElem {
    float A[N * N];
    float b[N];
    float C[sym_size(N)];
    float eta[N];
    float J[sym_size(N)];
};

// A prefix a_1 (x) ... (x) a_k has A = 0 (because A_1 = 0), so only its
// (b, C) = (filtered mean, filtered covariance) can reach any later result.
template <int N>
struct FState {
    float b[N];
    float C[sym_size(N)];
};

// Smoothing element of Lemma 5: a(x|z) = N(x; E z + g, L).
template <int N>
struct SElem {
    float E[N * N];
    float g[N];
    float L[sym_size(N)];
};

// A suffix a_k (x) ... (x) a_n has E = 0 (because E_n = 0): (g, L) are the
// smoothed mean and covariance.
template <int N>
struct SState {
    float g[N];
    float L[sym_size(N)];
};

// Per-model constants of the time-invariant case, computed once per call by
// the model-preparation kernel and kept in shared memory by the scans.
// For k > 1 Lemma 3's A_k, C_k, J_k do not depend on k; with the Cholesky
// factor S = L_S L_S^T of S = H Q H^T + R the element is carried as
//     J = U^T U,  eta_k = U^T w_k,  U = L_S^{-1} H F,  w_k = L_S^{-1} e_k,
//     b_k = u + K e_k,  e_k = y_k - H u - d,
// which is Lemma 3's J_k = F^T H^T S^{-1} H F and
// eta_k = F^T H^T S^{-1} (y_k - H u - d) factored through L_S.
template <int N, int M>
struct ModelConst {
    float F[N * N];
    float u[N];
    float Q[sym_size(N)];
    float A[N * N];         // (I - K H) F
    float C[sym_size(N)];   // Q - K S K^T  (= (I - K H) Q)
    float U[M * N];         // L_S^{-1} H F
    float K[N * M];         // Q H^T S^{-1}
    float Lsi[M * M];       // L_S^{-1} (lower triangular, row-major)
    float hud[M];           // H u + d
    float b1[N];            // k = 1 element (FP64-built): b_1
    float C1[sym_size(N)];  //                              C_1
    float pad[4];
};

// ---------------------------------------------------------------- helpers
template <int N>
KS_DEV void set_identity(FElem<N>& e) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) e.A[i * N + j] = (i == j) ? 1.f : 0.f;
        e.b[i] = 0.f;
        e.eta[i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < sym_size(N); ++i) { e.C[i] = 0.f; e.J[i] = 0.f; }
}

template <int N>
KS_DEV void set_identity(SElem<N>& e) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < N; ++j) e.E[i * N + j] = (i == j) ? 1.f : 0.f;
        e.g[i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < sym_size(N); ++i) e.L[i] = 0.f;
}

// Gauss-Jordan inverse with partial pivoting of an N x N register matrix.
// Row exchanges are done with selects so that no index is dynamic.
// Returns false when a pivot is not a finite non-zero number.
template <int N>
KS_DEV bool inverse_pp(float (&Mx)[N][N], float (&X)[N][N]) {
    bool ok = true;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) X[i][j] = (i == j) ? 1.f : 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        int p = k;
        float best = fabsf(Mx[k][k]);
#pragma unroll
        for (int r = k + 1; r < N; ++r) {
            float v = fabsf(Mx[r][k]);
            if (v > best) { best = v; p = r; }
        }
#pragma unroll
        for (int r = k + 1; r < N; ++r) {
            const bool s = (p == r);
#pragma unroll
            for (int c = 0; c < N; ++c) {
                float t = Mx[k][c];
                Mx[k][c] = s ? Mx[r][c] : t;
                Mx[r][c] = s ? t : Mx[r][c];
                float v = X[k][c];
                X[k][c] = s ? X[r][c] : v;
                X[r][c] = s ? v : X[r][c];
            }
        }
        const float piv = Mx[k][k];
        ok = ok && (fabsf(piv) > 1e-30f) && isfinite(piv);
        const float ip = __frcp_rn(piv);
#pragma unroll
        for (int c = 0; c < N; ++c) { Mx[k][c] *= ip; X[k][c] *= ip; }
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (r == k) continue;
            const float f = Mx[r][k];
#pragma unroll
            for (int c = 0; c < N; ++c) {
                Mx[r][c] = fmaf(-f, Mx[k][c], Mx[r][c]);
                X[r][c] = fmaf(-f, X[k][c], X[r][c]);
            }
        }
    }
    return ok;
}

// Column-sum (1-) norm of an N x N register matrix.
template <int N>
KS_DEV float norm1(const float (&X)[N][N]) {
    float m = 0.f;
#pragma unroll
    for (int c = 0; c < N; ++c) {
        float s = 0.f;
#pragma unroll
        for (int r = 0; r < N; ++r) s += fabsf(X[r][c]);
        m = fmaxf(m, s);
    }
    return m;
}

// One refinement step of X ~ M^{-1} for M = I + C J (C, J packed lower
// triangles, Lemma 4's I + C_i J_j), with the residual formed in FP64 from
// the FP32 inputs: row a of R = I - X M is e_a - x_a - (x_a C) J (x_a = row a
// of X), and X <- X + R X.
template <int N>
KS_DEV void refine_inverse_pp(const float (&C)[sym_size(N)], const float (&J)[sym_size(N)], float (&X)[N][N]) {
    float Xn[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        double v[N];
#pragma unroll
        for (int c = 0; c < N; ++c) {
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < N; ++k) t = fma((double)X[a][k], (double)C[sidx(k, c)], t);
            v[c] = t;
        }
        float r[N];
#pragma unroll
        for (int b = 0; b < N; ++b) {
            double t = (a == b ? 1.0 : 0.0) - (double)X[a][b];
#pragma unroll
            for (int c = 0; c < N; ++c) t = fma(-v[c], (double)J[sidx(c, b)], t);
            r[b] = (float)t;
        }
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float t = X[a][b];
#pragma unroll
            for (int k = 0; k < N; ++k) t = fmaf(r[k], X[k][b], t);
            Xn[a][b] = t;
        }
    }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) X[a][b] = Xn[a][b];
}

// Mi = (I + C J)^{-1} from Mx = I + C J (destroyed): FP32 Gauss-Jordan with
// partial pivoting, then one FP64-residual refinement step when the 1-norm
// condition estimate ||M||_1 ||Mi||_1 exceeds kRefineCond.  Returns FL_BAD on
// a failed pivot, FL_REFINED when the refinement ran, else 0.
template <int N, int REF = REF_FP64>
KS_DEV Flags inverse_cj(const float (&C)[sym_size(N)], const float (&J)[sym_size(N)], float (&Mx)[N][N],
                        float (&Mi)[N][N]) {
    if constexpr (REF == REF_NONE) return inverse_pp<N>(Mx, Mi) ? 0u : FL_BAD;
    const float nm = norm1<N>(Mx);
    if (!inverse_pp<N>(Mx, Mi)) return FL_BAD;
    const float cond = nm * norm1<N>(Mi);
    if (!(cond > kRefineCond) || !(cond < 3.0e38f)) return 0u;
    if constexpr (REF == REF_DETECT) {
        return FL_NEED;
    } else {
        refine_inverse_pp<N>(C, J, Mi);
        return FL_REFINED;
    }
}

// Cholesky G = L L^T of an M x M SPD matrix given as packed lower triangle;
// returns L^{-1} (lower, dense row-major).  G here is I + U C U^T >= I, so no
// pivoting is needed.  Returns false for a non-positive pivot.
template <int M>
KS_DEV bool chol_inv_lower(const float (&G)[sym_size(M)], float (&Li)[M][M]) {
    float Lc[M][M];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        float s = G[sidx(j, j)];
#pragma unroll
        for (int l = 0; l < j; ++l) s = fmaf(-Lc[j][l], Lc[j][l], s);
        ok = ok && (s > 0.f);
        const float r = rsqrtf(fmaxf(s, 1e-37f));
        Lc[j][j] = s * r;          // sqrt(s)
        Li[j][j] = r;              // 1 / L_jj
#pragma unroll
        for (int i = j + 1; i < M; ++i) {
            float t = G[sidx(i, j)];
#pragma unroll
            for (int l = 0; l < j; ++l) t = fmaf(-Lc[i][l], Lc[j][l], t);
            Lc[i][j] = t * r;
        }
#pragma unroll
        for (int i = 0; i < j; ++i) Lc[i][j] = 0.f;
    }
    // Li = Lc^{-1} by forward substitution, column by column.
#pragma unroll
    for (int c = 0; c < M; ++c) {
#pragma unroll
        for (int i = 0; i < M; ++i) {
            if (i < c) { Li[i][c] = 0.f; continue; }
            if (i == c) continue;
            float t = 0.f;
#pragma unroll
            for (int l = c; l < i; ++l) t = fmaf(-Lc[i][l], Li[l][c], t);
            Li[i][c] = t * Li[i][i];
        }
    }
    return ok;
}

// ---------------------------------------------------------------- Lemma 4
// General filtering operator, (A_i,..) (x) (A_j,..), with
//   M = I + C_i J_j,  Mi = M^{-1}  (one Gauss-Jordan inverse; (I + J_j C_i)^{-1}
//   = Mi^T because C_i, J_j are symmetric),
//   A_ij   = A_j Mi A_i
//   b_ij   = A_j Mi (b_i + C_i eta_j) + b_j
//   C_ij   = A_j (Mi C_i) A_j^T + C_j          (Mi C_i symmetric)
//   eta_ij = A_i^T Mi^T (eta_j - J_j b_i) + eta_i
//   J_ij   = A_i^T (Mi^T J_j) A_i + J_i       (Mi^T J_j symmetric)
template <int N, int REF = REF_FP64>
KS_DEV FElem<N> fcombine(const FElem<N>& ei, const FElem<N>& ej, Flags& bad) {
    FElem<N> r;
    float Mx[N][N], Mi[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float s = (a == b) ? 1.f : 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(ei.C[sidx(a, c)], ej.J[sidx(c, b)], s);
            Mx[a][b] = s;
        }
    bad |= inverse_cj<N, REF>(ei.C, ej.J, Mx, Mi);
    // X = A_j Mi
    float X[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(ej.A[a * N + c], Mi[c][b], s);
            X[a][b] = s;
        }
    // t = b_i + C_i eta_j ; b_ij = X t + b_j
    float t[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = ei.b[a];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(ei.C[sidx(a, c)], ej.eta[c], s);
        t[a] = s;
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = ej.b[a];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(X[a][c], t[c], s);
        r.b[a] = s;
    }
    // v = eta_j - J_j b_i ; w = Mi^T v ; eta_ij = A_i^T w + eta_i
    float v[N], w[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = ej.eta[a];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(-ej.J[sidx(a, c)], ei.b[c], s);
        v[a] = s;
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(Mi[c][a], v[c], s);
        w[a] = s;
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = ei.eta[a];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(ei.A[c * N + a], w[c], s);
        r.eta[a] = s;
    }
    // W = Mi C_i (lower) ; Y = A_j W ; C_ij = Y A_j^T + C_j (lower)
    float W[sym_size(N)];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(Mi[a][c], ei.C[sidx(c, b)], s);
            W[sidx(a, b)] = s;
        }
    {
        float Y[N][N];
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b < N; ++b) {
                float s = 0.f;
#pragma unroll
                for (int c = 0; c < N; ++c) s = fmaf(ej.A[a * N + c], W[sidx(c, b)], s);
                Y[a][b] = s;
            }
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) {
                float s = ej.C[sidx(a, b)];
#pragma unroll
                for (int c = 0; c < N; ++c) s = fmaf(Y[a][c], ej.A[b * N + c], s);
                r.C[sidx(a, b)] = s;
            }
    }
    // V = Mi^T J_j (lower) ; T1 = V A_i ; J_ij = A_i^T T1 + J_i (lower)
    {
        float V[sym_size(N)];
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) {
                float s = 0.f;
#pragma unroll
                for (int c = 0; c < N; ++c) s = fmaf(Mi[c][a], ej.J[sidx(c, b)], s);
                V[sidx(a, b)] = s;
            }
        float T1[N][N];
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b < N; ++b) {
                float s = 0.f;
#pragma unroll
                for (int c = 0; c < N; ++c) s = fmaf(V[sidx(a, c)], ei.A[c * N + b], s);
                T1[a][b] = s;
            }
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) {
                float s = ei.J[sidx(a, b)];
#pragma unroll
                for (int c = 0; c < N; ++c) s = fmaf(ei.A[c * N + a], T1[c][b], s);
                r.J[sidx(a, b)] = s;
            }
    }
    // A_ij = X A_i
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(X[a][c], ei.A[c * N + b], s);
            r.A[a * N + b] = s;
        }
    return r;
}

// Prefix (A = 0) combined with a general element: Lemma 4 with A_i = 0, of
// which only b and C are needed:
//   M = I + P J_j,  b' = A_j M^{-1} (xbar + P eta_j) + b_j,
//   C' = A_j (M^{-1} P) A_j^T + C_j.
template <int N, int REF = REF_FP64>
KS_DEV void fadvance(FState<N>& st, const FElem<N>& ej, Flags& bad) {
    float Mx[N][N], Mi[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float s = (a == b) ? 1.f : 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(st.C[sidx(a, c)], ej.J[sidx(c, b)], s);
            Mx[a][b] = s;
        }
    bad |= inverse_cj<N, REF>(st.C, ej.J, Mx, Mi);
    float t[N], mt[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = st.b[a];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(st.C[sidx(a, c)], ej.eta[c], s);
        t[a] = s;
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(Mi[a][c], t[c], s);
        mt[a] = s;
    }
    float W[sym_size(N)];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(Mi[a][c], st.C[sidx(c, b)], s);
            W[sidx(a, b)] = s;
        }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = ej.b[a];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(ej.A[a * N + c], mt[c], s);
        st.b[a] = s;
    }
    float Y[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(ej.A[a * N + c], W[sidx(c, b)], s);
            Y[a][b] = s;
        }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            float s = ej.C[sidx(a, b)];
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(Y[a][c], ej.A[b * N + c], s);
            st.C[sidx(a, b)] = s;
        }
}

// Rank-M form of Lemma 4 for a right operand that is a single measurement
// element (J_j = U^T U, eta_j = U^T w_j, A_j = A, C_j = C of ModelConst).
// With G = I_M + U C_i U^T = L L^T (SPD, >= I) the push-through identity gives
//   M^{-1}   = (I + C_i U^T U)^{-1} = I - CUL UL,   CUL = C_i U^T L^{-T}, UL = L^{-1} U
//   M^{-T} U^T = U^T G^{-1}
// so that, exactly as in Lemma 4,
//   A_ij   = A_j M^{-1} A_i,            b_ij = A_j M^{-1} (b_i + C_i U^T w_j) + b_j
//   C_ij   = A_j (C_i - CUL CUL^T) A_j^T + C_j
//   eta_ij = (UL A_i)^T L^{-1} (w_j - U b_i) + eta_i
//   J_ij   = (UL A_i)^T (UL A_i) + J_i
// with one M x M Cholesky factorisation instead of an N x N pivoted inverse.
// MC holds the element's A [N*N], C (packed lower) and U [M*N]: a ModelConst
// (time-invariant model) or one step's element of a time-varying model.
template <int N, int M, class MC>
KS_DEV FElem<N> fcombine_meas(const FElem<N>& ei, const MC& mc, const float (&bj)[N],
                              const float (&wj)[M], Flags& bad) {
    FElem<N> r;
    float CU[N][M];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int q = 0; q < M; ++q) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(ei.C[sidx(a, c)], mc.U[q * N + c], s);
            CU[a][q] = s;
        }
    float G[sym_size(M)];
#pragma unroll
    for (int q = 0; q < M; ++q)
#pragma unroll
        for (int p = 0; p <= q; ++p) {
            float s = (p == q) ? 1.f : 0.f;
#pragma unroll
            for (int a = 0; a < N; ++a) s = fmaf(mc.U[q * N + a], CU[a][p], s);
            G[sidx(q, p)] = s;
        }
    float Li[M][M];
    bad |= !chol_inv_lower<M>(G, Li);
    // CUL = CU Li^T (N x M),  UL = Li U (M x N)
    float CUL[N][M], UL[M][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int q = 0; q < M; ++q) {
            float s = 0.f;
#pragma unroll
            for (int p = 0; p <= q; ++p) s = fmaf(CU[a][p], Li[q][p], s);
            CUL[a][q] = s;
        }
#pragma unroll
    for (int q = 0; q < M; ++q)
#pragma unroll
        for (int a = 0; a < N; ++a) {
            float s = 0.f;
#pragma unroll
            for (int p = 0; p <= q; ++p) s = fmaf(Li[q][p], mc.U[p * N + a], s);
            UL[q][a] = s;
        }
    // X = A_j M^{-1} = A_j - (A_j CUL) UL
    float AC[N][M];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int q = 0; q < M; ++q) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(mc.A[a * N + c], CUL[c][q], s);
            AC[a][q] = s;
        }
    float X[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float s = mc.A[a * N + b];
#pragma unroll
            for (int q = 0; q < M; ++q) s = fmaf(-AC[a][q], UL[q][b], s);
            X[a][b] = s;
        }
    // b_ij = X (b_i + CU w_j) + b_j
    float t[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = ei.b[a];
#pragma unroll
        for (int q = 0; q < M; ++q) s = fmaf(CU[a][q], wj[q], s);
        t[a] = s;
    }
    float nb[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = bj[a];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(X[a][c], t[c], s);
        nb[a] = s;
    }
    // s = Li (w_j - U b_i) ; VA = UL A_i ; eta_ij = VA^T s + eta_i ; J_ij = VA^T VA + J_i
    float rr[M], sv[M];
#pragma unroll
    for (int q = 0; q < M; ++q) {
        float s = wj[q];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(-mc.U[q * N + c], ei.b[c], s);
        rr[q] = s;
    }
#pragma unroll
    for (int q = 0; q < M; ++q) {
        float s = 0.f;
#pragma unroll
        for (int p = 0; p <= q; ++p) s = fmaf(Li[q][p], rr[p], s);
        sv[q] = s;
    }
    float VA[M][N];
#pragma unroll
    for (int q = 0; q < M; ++q)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(UL[q][c], ei.A[c * N + b], s);
            VA[q][b] = s;
        }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = ei.eta[a];
#pragma unroll
        for (int q = 0; q < M; ++q) s = fmaf(VA[q][a], sv[q], s);
        r.eta[a] = s;
    }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            float s = ei.J[sidx(a, b)];
#pragma unroll
            for (int q = 0; q < M; ++q) s = fmaf(VA[q][a], VA[q][b], s);
            r.J[sidx(a, b)] = s;
        }
    // W = C_i - CUL CUL^T ; C_ij = A_j W A_j^T + C_j
    float W[sym_size(N)];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            float s = ei.C[sidx(a, b)];
#pragma unroll
            for (int q = 0; q < M; ++q) s = fmaf(-CUL[a][q], CUL[b][q], s);
            W[sidx(a, b)] = s;
        }
    {
        float Y[N][N];
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b < N; ++b) {
                float s = 0.f;
#pragma unroll
                for (int c = 0; c < N; ++c) s = fmaf(mc.A[a * N + c], W[sidx(c, b)], s);
                Y[a][b] = s;
            }
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) {
                float s = mc.C[sidx(a, b)];
#pragma unroll
                for (int c = 0; c < N; ++c) s = fmaf(Y[a][c], mc.A[b * N + c], s);
                r.C[sidx(a, b)] = s;
            }
    }
    float An[N * N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(X[a][c], ei.A[c * N + b], s);
            An[a * N + b] = s;
        }
#pragma unroll
    for (int a = 0; a < N * N; ++a) r.A[a] = An[a];
#pragma unroll
    for (int a = 0; a < N; ++a) r.b[a] = nb[a];
    return r;
}

// Prefix (A = 0) combined with a single measurement element (rank-M form):
//   b' = A_j M^{-1} (xbar + P U^T w_j) + b_j,   C' = A_j (P - CUL CUL^T) A_j^T + C_j.
template <int N, int M, class MC>
KS_DEV void fadvance_meas(FState<N>& st, const MC& mc, const float (&bj)[N],
                          const float (&wj)[M], Flags& bad) {
    float CU[N][M];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int q = 0; q < M; ++q) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(st.C[sidx(a, c)], mc.U[q * N + c], s);
            CU[a][q] = s;
        }
    float G[sym_size(M)];
#pragma unroll
    for (int q = 0; q < M; ++q)
#pragma unroll
        for (int p = 0; p <= q; ++p) {
            float s = (p == q) ? 1.f : 0.f;
#pragma unroll
            for (int a = 0; a < N; ++a) s = fmaf(mc.U[q * N + a], CU[a][p], s);
            G[sidx(q, p)] = s;
        }
    float Li[M][M];
    bad |= !chol_inv_lower<M>(G, Li);
    float CUL[N][M], UL[M][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int q = 0; q < M; ++q) {
            float s = 0.f;
#pragma unroll
            for (int p = 0; p <= q; ++p) s = fmaf(CU[a][p], Li[q][p], s);
            CUL[a][q] = s;
        }
#pragma unroll
    for (int q = 0; q < M; ++q)
#pragma unroll
        for (int a = 0; a < N; ++a) {
            float s = 0.f;
#pragma unroll
            for (int p = 0; p <= q; ++p) s = fmaf(Li[q][p], mc.U[p * N + a], s);
            UL[q][a] = s;
        }
    // t = xbar + CU w ; b' = A t - (A CUL)(UL t) + b_j
    float t[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = st.b[a];
#pragma unroll
        for (int q = 0; q < M; ++q) s = fmaf(CU[a][q], wj[q], s);
        t[a] = s;
    }
    float ult[M];
#pragma unroll
    for (int q = 0; q < M; ++q) {
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(UL[q][c], t[c], s);
        ult[q] = s;
    }
    float mt[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = t[a];
#pragma unroll
        for (int q = 0; q < M; ++q) s = fmaf(-CUL[a][q], ult[q], s);
        mt[a] = s;
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = bj[a];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(mc.A[a * N + c], mt[c], s);
        st.b[a] = s;
    }
    float W[sym_size(N)];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            float s = st.C[sidx(a, b)];
#pragma unroll
            for (int q = 0; q < M; ++q) s = fmaf(-CUL[a][q], CUL[b][q], s);
            W[sidx(a, b)] = s;
        }
    float Y[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(mc.A[a * N + c], W[sidx(c, b)], s);
            Y[a][b] = s;
        }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            float s = mc.C[sidx(a, b)];
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(Y[a][c], mc.A[b * N + c], s);
            st.C[sidx(a, b)] = s;
        }
}

// Lemma 3 element for k > 1 from one measurement: e = y - H u - d,
// b = u + K e, w = L_S^{-1} e (eta = U^T w, J = U^T U are implied).
template <int N, int M>
KS_DEV void meas_element(const ModelConst<N, M>& mc, const float (&y)[M], float (&b)[N],
                         float (&w)[M]) {
    float e[M];
#pragma unroll
    for (int q = 0; q < M; ++q) e[q] = y[q] - mc.hud[q];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = mc.u[a];
#pragma unroll
        for (int q = 0; q < M; ++q) s = fmaf(mc.K[a * M + q], e[q], s);
        b[a] = s;
    }
#pragma unroll
    for (int q = 0; q < M; ++q) {
        float s = 0.f;
#pragma unroll
        for (int p = 0; p <= q; ++p) s = fmaf(mc.Lsi[q * M + p], e[p], s);
        w[q] = s;
    }
}

// The same element expanded to the general form (A, b, C, eta, J).
template <int N, int M, class MC>
KS_DEV void expand_meas(const MC& mc, const float (&b)[N], const float (&w)[M],
                        FElem<N>& e) {
#pragma unroll
    for (int a = 0; a < N * N; ++a) e.A[a] = mc.A[a];
#pragma unroll
    for (int a = 0; a < sym_size(N); ++a) e.C[a] = mc.C[a];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        e.b[a] = b[a];
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < M; ++q) s = fmaf(mc.U[q * N + a], w[q], s);
        e.eta[a] = s;
    }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b2 = 0; b2 <= a; ++b2) {
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < M; ++q) s = fmaf(mc.U[q * N + a], mc.U[q * N + b2], s);
            e.J[sidx(a, b2)] = s;
        }
}

// The k = 1 element of Lemma 3: A_1 = 0, (b_1, C_1) built in FP64, eta_1 = J_1 = 0.
template <int N, int M>
KS_DEV void first_element(const ModelConst<N, M>& mc, FElem<N>& e) {
#pragma unroll
    for (int a = 0; a < N * N; ++a) e.A[a] = 0.f;
#pragma unroll
    for (int a = 0; a < N; ++a) { e.b[a] = mc.b1[a]; e.eta[a] = 0.f; }
#pragma unroll
    for (int a = 0; a < sym_size(N); ++a) { e.C[a] = mc.C1[a]; e.J[a] = 0.f; }
}

// ---------------------------------------------------------------- linear block fold
// For a time-invariant model every measurement element has the same A, C,
// J = U^T U (Lemma 3: only b_k and eta_k depend on k), so the fold of a block
// of l consecutive measurement elements, a_1 (x) ... (x) a_l (Lemma 4), has the
// same A, C, J for every block, and its (b, eta) is affine in the block's
// measurements: the rank-ny combine maps (b, eta) of the running aggregate and
// of the next element linearly, with coefficients that depend only on the
// matrices.  BlockCoef holds, for blocks of `ch` steps,
//   b   = bc + Bs y_0 + sum_{i>0} Bc[i] (y_i - y_0),
//   eta = ec + Es y_0 + sum_{i>0} Ec[i] (y_i - y_0),
// and the block's A, C, J.  Writing the measurements relative to the block's
// first one keeps the products small where y is large.  Bs (= sum_i Bc[i])
// then multiplies the large y_0, and the scan adds Bs y_0 to A x_prev, which
// nearly cancels it in the directions that y tracks; Bs is therefore formed
// from the block's own A and J rather than summed (see block_coef_warp), so
// that the cancellation is as exact as in the element-by-element fold.  The
// scans fold a full block with it in 2 N M FMAs per step instead of one rank-ny
// combine; blocks that hold a sequence's first step, or a ragged end, fold
// element by element.
template <int N, int M>
struct alignas(16) BlockCoef {
    float Bc[32][N * M];   // position i: row-major N x M
    float Ec[32][N * M];
    float Bs[N * M], Es[N * M];   // coefficients of y_0
    float bc[N], ec[N];
    float A[N * N];
    float C[sym_size(N)];
    float J[sym_size(N)];
    int ch;                // block length the coefficients are for (0: none)
    int pad[3];
};

// Coefficients of blocks of `ch` steps (a power of two, <= 32), by one warp,
// by doubling: a block of 2h steps is the Lemma 4 combine of two blocks of h
// steps, whose matrix parts (A_h, C_h, J_h) are the same.  Every lane runs the
// matrix combines (the same values; five levels for 32 steps), and lane i
// keeps the coefficients of position i within its current block.  With
// M = I + C_h J_h, P = A_h M^{-1}, R = A_h^T M^{-T}:
//   b = P (b_L + C_h eta_R) + b_R,   eta = R (eta_R - J_h b_L) + eta_L,
// so a position of the left half maps as Bc <- P Bc, Ec <- Ec - R J_h Bc, and
// one of the right half as Bc <- P C_h Ec + Bc, Ec <- R Ec.  A block of one
// step is the measurement element: A, C, J = U^T U, Bc = K, Ec = U^T L_S^{-1}.
//
// The terms in y_0 follow from a noise-free trajectory.  For any state z, the
// measurements ybar_i = H x_i + d of the trajectory x_i = F x_{i-1} + u from
// x_prev = z (no noise) are their own prior means, so the block's posterior
// mean of x_end given x_prev = z is the trajectory's end, and the likelihood's
// information vector is J z:  b(ybar) = x_end - A z,  eta(ybar) = J z.  With
// b, eta affine in y and z = L y_0,
//   b = x_end - A L y_0 + sum_i Bc[i] (y_i - ybar_i),
//   eta = J L y_0 + sum_i Ec[i] (y_i - ybar_i),
// where ybar_i = G_i y_0 + g_i, G_i = H F^{i+1} L, g_i = H c_{i+1} + d,
// c_j = sum_{l<j} F^l u, x_end = F^ch L y_0 + c_ch.  This holds for any L;
// L = H^T (H H^T)^{-1} puts z on the measured components, and where y follows
// a stationary direction of F (the positions of a tracking model) then
// ybar_i = y_0, G_i = I, and Bs = F^ch L - A L, made of the same A the scan
// multiplies x_prev with.  Lane i forms F^{i+1} L and c_{i+1} from the powers
// F^h, c_h by the bits of i + 1; the sums over positions are warp reductions.
// `ch` = 0 is written when an inverse fails (then the scans fold element by
// element).
template <int N, int M>
KS_DEV void block_coef_warp(const ModelConst<N, M>& mc, const float* __restrict__ Hs, int ch,
                            BlockCoef<N, M>* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    float Ah[N][N], Ch[N][N], Jh[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            Ah[a][b] = mc.A[a * N + b];
            Ch[a][b] = mc.C[sidx(a, b)];
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < M; ++q) s = fmaf(mc.U[q * N + a], mc.U[q * N + b], s);
            Jh[a][b] = s;
        }
    float Bc[N][M], Ec[N][M];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int r = 0; r < M; ++r) {
            Bc[a][r] = mc.K[a * M + r];
            float s = 0.f;   // U^T L_S^{-1}
#pragma unroll
            for (int q = r; q < M; ++q) s = fmaf(mc.U[q * N + a], mc.Lsi[q * M + r], s);
            Ec[a][r] = s;
        }
    bool ok = ch >= 1 && ch <= 32 && (ch & (ch - 1)) == 0;
#pragma unroll 1
    for (int h = 1; ok && h < ch; h <<= 1) {
        float Mx[N][N], Mi[N][N];
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b < N; ++b) {
                float s = (a == b) ? 1.f : 0.f;
#pragma unroll
                for (int c = 0; c < N; ++c) s = fmaf(Ch[a][c], Jh[c][b], s);
                Mx[a][b] = s;
            }
        ok = inverse_pp<N>(Mx, Mi);
        float P[N][N], Rt[N][N], PC[N][N], RJ[N][N];   // Rt = R^T = M^{-1} A_h
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b < N; ++b) {
                float s = 0.f, t = 0.f;
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    s = fmaf(Ah[a][c], Mi[c][b], s);
                    t = fmaf(Mi[a][c], Ah[c][b], t);
                }
                P[a][b] = s;
                Rt[a][b] = t;
            }
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b < N; ++b) {
                float s = 0.f, t = 0.f;
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    s = fmaf(P[a][c], Ch[c][b], s);
                    t = fmaf(Rt[c][a], Jh[c][b], t);   // (R J_h)[a][b], R = Rt^T
                }
                PC[a][b] = s;
                RJ[a][b] = t;
            }
        // this lane's position: left or right half of the new block of 2h
        const bool right = (lane & h) != 0;
        {
            float nB[N][M], nE[N][M];
#pragma unroll
            for (int a = 0; a < N; ++a)
#pragma unroll
                for (int r = 0; r < M; ++r) {
                    float sb, se;
                    if (!right) {
                        sb = 0.f;
                        se = Ec[a][r];
#pragma unroll
                        for (int c = 0; c < N; ++c) {
                            sb = fmaf(P[a][c], Bc[c][r], sb);
                            se = fmaf(-RJ[a][c], Bc[c][r], se);
                        }
                    } else {
                        sb = Bc[a][r];
                        se = 0.f;
#pragma unroll
                        for (int c = 0; c < N; ++c) {
                            sb = fmaf(PC[a][c], Ec[c][r], sb);
                            se = fmaf(Rt[c][a], Ec[c][r], se);
                        }
                    }
                    nB[a][r] = sb;
                    nE[a][r] = se;
                }
#pragma unroll
            for (int a = 0; a < N; ++a)
#pragma unroll
                for (int r = 0; r < M; ++r) { Bc[a][r] = nB[a][r]; Ec[a][r] = nE[a][r]; }
        }
        {   // matrix part: A <- P A_h, C <- P C_h A_h^T + C_h, J <- A_h^T M^{-T} J_h A_h + J_h
            float nA[N][N], nC[N][N], nJ[N][N];
#pragma unroll
            for (int a = 0; a < N; ++a)
#pragma unroll
                for (int b = 0; b < N; ++b) {
                    float sa = 0.f, sc = Ch[a][b], sj = Jh[a][b];
#pragma unroll
                    for (int c = 0; c < N; ++c) {
                        sa = fmaf(P[a][c], Ah[c][b], sa);
                        sc = fmaf(PC[a][c], Ah[b][c], sc);
                        sj = fmaf(RJ[a][c], Ah[c][b], sj);
                    }
                    nA[a][b] = sa;
                    nC[a][b] = sc;
                    nJ[a][b] = sj;
                }
#pragma unroll
            for (int a = 0; a < N; ++a)
#pragma unroll
                for (int b = 0; b < N; ++b) {
                    Ah[a][b] = nA[a][b];
                    Ch[a][b] = 0.5f * (nC[a][b] + nC[b][a]);
                    Jh[a][b] = 0.5f * (nJ[a][b] + nJ[b][a]);
                }
        }
    }
    if (lane < ch) {
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int r = 0; r < M; ++r) {
                out->Bc[lane][a * M + r] = Bc[a][r];
                out->Ec[lane][a * M + r] = Ec[a][r];
            }
    }
    // ---- the lift L = H^T (H H^T)^{-1} (0 if H H^T is singular) and A L, J L
    float Lf[N][M], AL[N][M], JL[N][M];
    {
        float G[M][M], Gi[M][M];
#pragma unroll
        for (int q = 0; q < M; ++q)
#pragma unroll
            for (int r = 0; r < M; ++r) {
                float s = 0.f;
#pragma unroll
                for (int c = 0; c < N; ++c) s = fmaf(Hs[q * N + c], Hs[r * N + c], s);
                G[q][r] = s;
            }
        const bool lift = inverse_pp<M>(G, Gi);
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int r = 0; r < M; ++r) {
                float s = 0.f;
#pragma unroll
                for (int q = 0; q < M; ++q) s = fmaf(Hs[q * N + a], Gi[q][r], s);
                Lf[a][r] = lift ? s : 0.f;
            }
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int r = 0; r < M; ++r) {
                float s = 0.f, t = 0.f;
#pragma unroll
                for (int c = 0; c < N; ++c) {
                    s = fmaf(Ah[a][c], Lf[c][r], s);
                    t = fmaf(Jh[a][c], Lf[c][r], t);
                }
                AL[a][r] = s;
                JL[a][r] = t;
            }
    }
    if (lane == 0) {
#pragma unroll
        for (int a = 0; a < N; ++a) {
#pragma unroll
            for (int b = 0; b < N; ++b) out->A[a * N + b] = Ah[a][b];
#pragma unroll
            for (int b = 0; b <= a; ++b) { out->C[sidx(a, b)] = Ch[a][b]; out->J[sidx(a, b)] = Jh[a][b]; }
        }
    }
    // ---- lane i: V = F^{i+1} L and c = c_{i+1}, from (F^h, c_h) by the bits of i + 1
    float V[N][M], cv[N];
    {
        float Fp[N][N], cp[N];
#pragma unroll
        for (int a = 0; a < N; ++a) {
            cv[a] = 0.f;
            cp[a] = mc.u[a];
#pragma unroll
            for (int b = 0; b < N; ++b) Fp[a][b] = mc.F[a * N + b];
#pragma unroll
            for (int r = 0; r < M; ++r) V[a][r] = Lf[a][r];
        }
        const int j = lane + 1;
#pragma unroll 1
        for (int h = 1; h <= ch; h <<= 1) {
            if (j & h) {
                float nV[N][M], nc[N];
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    float s = cp[a];
#pragma unroll
                    for (int c = 0; c < N; ++c) s = fmaf(Fp[a][c], cv[c], s);
                    nc[a] = s;
#pragma unroll
                    for (int r = 0; r < M; ++r) {
                        float t = 0.f;
#pragma unroll
                        for (int c = 0; c < N; ++c) t = fmaf(Fp[a][c], V[c][r], t);
                        nV[a][r] = t;
                    }
                }
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    cv[a] = nc[a];
#pragma unroll
                    for (int r = 0; r < M; ++r) V[a][r] = nV[a][r];
                }
            }
            if (2 * h <= ch) {   // (F^2h, c_2h) = (F^h F^h, F^h c_h + c_h)
                float nF[N][N], nc[N];
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    float s = cp[a];
#pragma unroll
                    for (int c = 0; c < N; ++c) s = fmaf(Fp[a][c], cp[c], s);
                    nc[a] = s;
#pragma unroll
                    for (int b = 0; b < N; ++b) {
                        float t = 0.f;
#pragma unroll
                        for (int c = 0; c < N; ++c) t = fmaf(Fp[a][c], Fp[c][b], t);
                        nF[a][b] = t;
                    }
                }
#pragma unroll
                for (int a = 0; a < N; ++a) {
                    cp[a] = nc[a];
#pragma unroll
                    for (int b = 0; b < N; ++b) Fp[a][b] = nF[a][b];
                }
            }
        }
    }
    // ---- this position's ybar_i - y_0 = (G_i - I) y_0 + g_i and its terms
    const bool in = lane < ch;
    float tB[N][M], tE[N][M], tb[N], te[N];
    {
        float Gm[M][M], g[M];
#pragma unroll
        for (int q = 0; q < M; ++q) {
            float s = mc.hud[q];   // H c_{i+1} + d = H u + d + H (c_{i+1} - u)
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(Hs[q * N + c], cv[c] - mc.u[c], s);
            g[q] = s;
#pragma unroll
            for (int r = 0; r < M; ++r) {
                float t = (q == r) ? -1.f : 0.f;
#pragma unroll
                for (int c = 0; c < N; ++c) t = fmaf(Hs[q * N + c], V[c][r], t);
                Gm[q][r] = t;
            }
        }
#pragma unroll
        for (int a = 0; a < N; ++a) {
            float sb = 0.f, se = 0.f;
#pragma unroll
            for (int q = 0; q < M; ++q) {
                sb = fmaf(Bc[a][q], g[q], sb);
                se = fmaf(Ec[a][q], g[q], se);
            }
            tb[a] = in ? sb : 0.f;
            te[a] = in ? se : 0.f;
#pragma unroll
            for (int r = 0; r < M; ++r) {
                float s = 0.f, t = 0.f;
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    s = fmaf(Bc[a][q], Gm[q][r], s);
                    t = fmaf(Ec[a][q], Gm[q][r], t);
                }
                tB[a][r] = in ? s : 0.f;
                tE[a][r] = in ? t : 0.f;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int a = 0; a < N; ++a) {
            tb[a] += __shfl_xor_sync(0xffffffffu, tb[a], o);
            te[a] += __shfl_xor_sync(0xffffffffu, te[a], o);
#pragma unroll
            for (int r = 0; r < M; ++r) {
                tB[a][r] += __shfl_xor_sync(0xffffffffu, tB[a][r], o);
                tE[a][r] += __shfl_xor_sync(0xffffffffu, tE[a][r], o);
            }
        }
    }
    // ---- x_end = F^ch L y_0 + c_ch from the block's last position
    const int last = (ch >= 1 && ch <= 32) ? ch - 1 : 0;
#pragma unroll
    for (int a = 0; a < N; ++a) {
        const float w = __shfl_sync(0xffffffffu, cv[a], last);
        if (lane == 0) {
            out->bc[a] = w - tb[a];
            out->ec[a] = -te[a];
        }
#pragma unroll
        for (int r = 0; r < M; ++r) {
            const float W = __shfl_sync(0xffffffffu, V[a][r], last);
            if (lane == 0) {
                out->Bs[a * M + r] = (W - AL[a][r]) - tB[a][r];
                out->Es[a * M + r] = JL[a][r] - tE[a][r];
            }
        }
    }
    if (lane == 0) {
        out->ch = ok ? ch : 0;
    }
}

// ---------------------------------------------------------------- Lemma 5
// Smoothing element for k < n from the filtered (xbar, P):
//   P- = F P F^T + Q = Lc Lc^T (Cholesky),  E = P F^T (P-)^{-1}  (solved as
//   E^T = (P-)^{-1} (F P)),  g = xbar - E (F xbar + u),  L = P - E (F P).
// MC holds F [N*N], u [N] and Q (packed lower): a ModelConst, or one step's
// transition of a time-varying model.
template <int N, int M, class MC, class FL>
KS_DEV void smoother_element(const MC& mc, const float (&xbar)[N],
                             const float (&P)[sym_size(N)], SElem<N>& e, FL& bad) {
    float FP[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(mc.F[a * N + c], P[sidx(c, b)], s);
            FP[a][b] = s;
        }
    float Lc[N][N];
    float rd[N];
    {
        float Pm[sym_size(N)];
#pragma unroll
        for (int a = 0; a < N; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) {
                float s = mc.Q[sidx(a, b)];
#pragma unroll
                for (int c = 0; c < N; ++c) s = fmaf(FP[a][c], mc.F[b * N + c], s);
                Pm[sidx(a, b)] = s;
            }
#pragma unroll
        for (int j = 0; j < N; ++j) {
            float s = Pm[sidx(j, j)];
#pragma unroll
            for (int l = 0; l < j; ++l) s = fmaf(-Lc[j][l], Lc[j][l], s);
            bad |= !(s > 0.f);
            const float r = rsqrtf(fmaxf(s, 1e-37f));
            Lc[j][j] = s * r;
            rd[j] = r;
#pragma unroll
            for (int i = j + 1; i < N; ++i) {
                float t = Pm[sidx(i, j)];
#pragma unroll
                for (int l = 0; l < j; ++l) t = fmaf(-Lc[i][l], Lc[j][l], t);
                Lc[i][j] = t * r;
            }
        }
    }
    // Solve Lc Lc^T X = FP for X = E^T, column by column.
    float X[N][N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            float t = FP[i][c];
#pragma unroll
            for (int l = 0; l < i; ++l) t = fmaf(-Lc[i][l], X[l][c], t);
            X[i][c] = t * rd[i];
        }
#pragma unroll
        for (int i = N - 1; i >= 0; --i) {
            float t = X[i][c];
#pragma unroll
            for (int l = i + 1; l < N; ++l) t = fmaf(-Lc[l][i], X[l][c], t);
            X[i][c] = t * rd[i];
        }
    }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) e.E[a * N + b] = X[b][a];
    // g = xbar - E (F xbar + u)
    float fx[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = mc.u[a];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(mc.F[a * N + c], xbar[c], s);
        fx[a] = s;
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = xbar[a];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(-e.E[a * N + c], fx[c], s);
        e.g[a] = s;
    }
    // L = P - E (F P)  (lower)
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            float s = P[sidx(a, b)];
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(-e.E[a * N + c], FP[c][b], s);
            e.L[sidx(a, b)] = s;
        }
}

// ---------------------------------------------------------------- Lemma 6
// a_i (x) a_j with a_i the earlier time step:
//   E_ij = E_i E_j,  g_ij = E_i g_j + g_i,  L_ij = E_i L_j E_i^T + L_i.
template <int N>
KS_DEV SElem<N> scombine(const SElem<N>& ei, const SElem<N>& ej) {
    SElem<N> r;
    float Y[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(ei.E[a * N + c], ej.L[sidx(c, b)], s);
            Y[a][b] = s;
        }
    float nL[sym_size(N)], ng[N], nE[N * N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            float s = ei.L[sidx(a, b)];
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(Y[a][c], ei.E[b * N + c], s);
            nL[sidx(a, b)] = s;
        }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = ei.g[a];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(ei.E[a * N + c], ej.g[c], s);
        ng[a] = s;
    }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(ei.E[a * N + c], ej.E[c * N + b], s);
            nE[a * N + b] = s;
        }
#pragma unroll
    for (int a = 0; a < N * N; ++a) r.E[a] = nE[a];
#pragma unroll
    for (int a = 0; a < N; ++a) r.g[a] = ng[a];
#pragma unroll
    for (int a = 0; a < sym_size(N); ++a) r.L[a] = nL[a];
    return r;
}

// a_i (x) suffix (E = 0): g = E_i g_s + g_i,  L = E_i L_s E_i^T + L_i.
template <int N>
KS_DEV void sadvance(const SElem<N>& ei, SState<N>& st) {
    float Y[N][N];
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b < N; ++b) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(ei.E[a * N + c], st.L[sidx(c, b)], s);
            Y[a][b] = s;
        }
    float ng[N];
#pragma unroll
    for (int a = 0; a < N; ++a) {
        float s = ei.g[a];
#pragma unroll
        for (int c = 0; c < N; ++c) s = fmaf(ei.E[a * N + c], st.g[c], s);
        ng[a] = s;
    }
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) {
            float s = ei.L[sidx(a, b)];
#pragma unroll
            for (int c = 0; c < N; ++c) s = fmaf(Y[a][c], ei.E[b * N + c], s);
            st.L[sidx(a, b)] = s;
        }
#pragma unroll
    for (int a = 0; a < N; ++a) st.g[a] = ng[a];
}

}  // namespace ks
