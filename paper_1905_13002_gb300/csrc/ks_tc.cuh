// ks_tc.cuh -- Lemma 3-6 operators for nx = 32 with their dense products on
// the tensor cores (one warp per chain of time steps).
//
// Every 32 x 32 x {32, ny} product runs as warp-level mma.sync m16n8k8 TF32
// instructions in the 3xTF32 form: each FP32 operand x is split x = hi + lo
// with hi = tf32(x) and lo = tf32(x - hi), and a b is accumulated in FP32 as
// a_hi b_hi + (a_lo b_hi + a_hi b_lo), the two parts in separate accumulators
// (a_lo b_lo is below FP32 resolution and dropped).  Operands and results are
// row-major matrices in shared memory with a row pitch of 36 floats, so that
// ldmatrix row reads and fragment loads hit distinct banks.
//
// Elements are sets of pointers into a per-warp pool of matrix buffers; each
// buffer is 32 rows plus one vector row (b with C, eta with J, g with L), so an
// operator can update a matrix in place or hand a fresh buffer to its result
// without copying.  Symmetric results (C, J, L) are symmetrised in place.
//
// The pivoted inverse (Gauss-Jordan, in place, lane r holding one row of the
// transposed matrix) runs on the CUDA cores.  When the 1-norm condition
// estimate ||M||_1 ||M^{-1}||_1 exceeds kRefineCond the inverse gets one step of
// refinement, X <- X + X R with the residual R = I - M X formed in FP64.
#pragma once

#include "ks_ops.cuh"

namespace ks {
namespace tc {

constexpr unsigned kFull = 0xffffffffu;

// Unrolling of the k loop of the tensor-core products (code size against
// cross-step scheduling).
#ifndef KS_TC_KT_UNROLL
#define KS_TC_KT_UNROLL 2
#endif
constexpr int kMmUnroll = KS_TC_KT_UNROLL;

template <int N>
struct TD {
    static_assert(N == 32, "the tensor-core operators hold one row per lane");
    static constexpr int P = N + 4;            // row pitch (floats)
    static constexpr int MAT = (N + 1) * P;    // one buffer: N rows + a vector row
};

template <int N>
KS_DEV float* vrow(float* m) { return m + N * TD<N>::P; }
template <int N>
KS_DEV const float* vrow(const float* m) { return m + N * TD<N>::P; }

KS_DEV int lane_id() { return threadIdx.x & 31; }

// Per-warp pool of matrix buffers (a bit mask of the free ones; every lane
// holds the same mask).  An empty pool is a logic error: it is reported
// through `bad` and hands out the first buffer, which stays in bounds.
template <int N>
struct Pool {
    float* base;
    uint32_t mask;
    KS_DEV float* get(Flags& bad) {
        if (mask == 0u) {
            bad |= FL_BAD;
            return base;
        }
        const int i = __ffs(mask) - 1;
        mask &= mask - 1u;
        return base + i * TD<N>::MAT;
    }
    KS_DEV void put(const float* p) {
        if (p) mask |= 1u << (int)((p - base) / TD<N>::MAT);
    }
};

// Filtering element (Lemma 3/4): b in the vector row of C, eta in that of J.
struct FE {
    float *A, *C, *J;
};
// Smoothing element (Lemma 5/6): g in the vector row of L.
struct SE {
    float *E, *L;
};

// ---------------------------------------------------------------- tensor-core primitives
KS_DEV uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

KS_DEV uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
// x = hi + lo with hi = tf32(x) rounded to nearest; lo = x - hi is exact in
// FP32 and handed over as is (the tensor core reads its top 19 bits).
KS_DEV void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = to_tf32(x);
    lo = __float_as_uint(x - __uint_as_float(hi));
}
KS_DEV void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// ldmatrix on 32-bit data: an 8 x 8 b16 tile is an 8 x 4 float tile, and lane
// t receives the float at (t / 4, t % 4) of it.
KS_DEV void ldsm_x4(uint32_t (&r)[4], const float* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p))
                 : "memory");
}
KS_DEV void ldsm_x2(uint32_t (&r)[2], const float* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(smem_u32(p))
                 : "memory");
}

// C = sa op(A) op(B) (+ D), shared-memory matrices of row pitch PP.
// op(A)(i, k) = TA ? A[k][i] : A[i][k];  op(B)(k, n) = TB ? B[n][k] : B[k][n].
// MM x KK times KK x NN, MM a multiple of 16, NN and KK of 8.  C must not
// alias A or B; it may equal D (each output element reads only its own D).
// Row-major A and transposed B go through ldmatrix.  The k loop is outermost
// and every output tile keeps its two accumulators (hi*hi and the cross terms)
// live, so each k step issues 3 MT NT independent mma.  Ends with a warp
// barrier.
template <int MM, int NN, int KK, int PP, bool TA, bool TB>
KS_DEV void mm(const float* A, const float* B, float* C, const float* D = nullptr, float sa = 1.f) {
    static_assert(MM % 16 == 0 && NN % 8 == 0 && KK % 8 == 0, "tile shape");
    constexpr int MT = MM / 16, NT = NN / 8, KT = KK / 8;
    const int lane = lane_id(), gid = lane >> 2, tig = lane & 3;
    float big[MT][NT][4], sml[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) big[mt][nt][e] = sml[mt][nt][e] = 0.f;
#pragma unroll kMmUnroll
    for (int kt = 0; kt < KT; ++kt) {
        const int k0 = kt * 8;
        uint32_t ah[MT][4], al[MT][4], bh[NT][2], bl[NT][2];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            const int i0 = mt * 16;
            float a[4];
            if constexpr (!TA) {
                uint32_t q4[4];
                const int q = lane >> 3, rr = lane & 7;
                ldsm_x4(q4, A + (i0 + rr + (q & 1) * 8) * PP + k0 + (q >> 1) * 4);
#pragma unroll
                for (int e = 0; e < 4; ++e) a[e] = __uint_as_float(q4[e]);
            } else {
                a[0] = A[(k0 + tig) * PP + i0 + gid];
                a[1] = A[(k0 + tig) * PP + i0 + gid + 8];
                a[2] = A[(k0 + tig + 4) * PP + i0 + gid];
                a[3] = A[(k0 + tig + 4) * PP + i0 + gid + 8];
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) split_tf32(sa * a[e], ah[mt][e], al[mt][e]);
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const int n0 = nt * 8;
            float b[2];
            if constexpr (TB) {
                if (NT % 2 == 0) {
                    if (nt % 2 == 1) continue;       // loaded with the even tile
                    uint32_t q4[4];
                    const int q = lane >> 3, rr = lane & 7;
                    ldsm_x4(q4, B + (n0 + (q >> 1) * 8 + rr) * PP + k0 + (q & 1) * 4);
                    split_tf32(__uint_as_float(q4[0]), bh[nt][0], bl[nt][0]);
                    split_tf32(__uint_as_float(q4[1]), bh[nt][1], bl[nt][1]);
                    split_tf32(__uint_as_float(q4[2]), bh[nt + 1][0], bl[nt + 1][0]);
                    split_tf32(__uint_as_float(q4[3]), bh[nt + 1][1], bl[nt + 1][1]);
                    continue;
                }
                uint32_t q2[2];
                const int q = (lane >> 3) & 1, rr = lane & 7;
                ldsm_x2(q2, B + (n0 + rr) * PP + k0 + q * 4);
                b[0] = __uint_as_float(q2[0]);
                b[1] = __uint_as_float(q2[1]);
            } else {
                b[0] = B[(k0 + tig) * PP + n0 + gid];
                b[1] = B[(k0 + tig + 4) * PP + n0 + gid];
            }
            split_tf32(b[0], bh[nt][0], bl[nt][0]);
            split_tf32(b[1], bh[nt][1], bl[nt][1]);
        }
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                mma_tf32(sml[mt][nt], al[mt], bh[nt]);
                mma_tf32(sml[mt][nt], ah[mt], bl[nt]);
                mma_tf32(big[mt][nt], ah[mt], bh[nt]);
            }
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const int r0 = mt * 16 + gid, c0 = nt * 8 + 2 * tig;
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = big[mt][nt][e] + sml[mt][nt][e];
            if (D) {
                const float2 d0 = *reinterpret_cast<const float2*>(D + r0 * PP + c0);
                const float2 d1 = *reinterpret_cast<const float2*>(D + (r0 + 8) * PP + c0);
                v[0] += d0.x;
                v[1] += d0.y;
                v[2] += d1.x;
                v[3] += d1.y;
            }
            *reinterpret_cast<float2*>(C + r0 * PP + c0) = make_float2(v[0], v[1]);
            *reinterpret_cast<float2*>(C + (r0 + 8) * PP + c0) = make_float2(v[2], v[3]);
        }
    __syncwarp();
}

template <int N, bool TA, bool TB>
KS_DEV void mmq(const float* A, const float* B, float* C, const float* D = nullptr, float sa = 1.f) {
    mm<N, N, N, TD<N>::P, TA, TB>(A, B, C, D, sa);
}

// ---------------------------------------------------------------- vector and layout helpers
// sum_c X[r][c] v[c], visiting the columns from c = r on so that the warp's
// loads of X fall on distinct banks.
template <int N>
KS_DEV float rdot(const float* X, int r, const float* v) {
    float s = 0.f;
#pragma unroll 8
    for (int d = 0; d < N; ++d) {
        const int c = (r + d) & (N - 1);
        s = fmaf(X[r * TD<N>::P + c], v[c], s);
    }
    return s;
}
// sum_k X[k][r] v[k]
template <int N>
KS_DEV float cdot(const float* X, int r, const float* v) {
    float s = 0.f;
#pragma unroll 8
    for (int k = 0; k < N; ++k) s = fmaf(X[k * TD<N>::P + r], v[k], s);
    return s;
}
template <int N>
KS_DEV void add_diag(float* X, float v) {
    const int r = lane_id();
    X[r * TD<N>::P + r] += v;
    __syncwarp();
}
// X <- (X + X^T) / 2 in place: lane r owns the pairs (r, r + d), d = 1..N/2
// (d = N/2 for r < N/2 only), so every element is written once.
template <int N>
KS_DEV void symm(float* X) {
    constexpr int P = TD<N>::P;
    const int r = lane_id();
#pragma unroll 4
    for (int d = 1; d <= N / 2; ++d) {
        const int c = (r + d) & (N - 1);
        if (d < N / 2 || r < N / 2) {
            const float m = 0.5f * (X[r * P + c] + X[c * P + r]);
            X[r * P + c] = m;
            X[c * P + r] = m;
        }
    }
    __syncwarp();
}
template <int N>
KS_DEV void zero_mat(float* X) {
    const int r = lane_id();
#pragma unroll 8
    for (int q = 0; q < N; ++q) X[q * TD<N>::P + r] = 0.f;
    __syncwarp();
}
template <int N>
KS_DEV void copy_mat(float* dst, const float* src) {
    const int r = lane_id();
#pragma unroll 8
    for (int q = 0; q < N; ++q) dst[q * TD<N>::P + r] = src[q * TD<N>::P + r];
    __syncwarp();
}

// Global <-> shared.  Global matrices are dense N x N row-major (16-byte
// aligned); loads go through cp.async (L2, no register staging) and are
// completed by cp_wait().
KS_DEV void cp16(float* sdst, const float* gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(sdst)), "l"(gsrc) : "memory");
}
KS_DEV void cp_wait() {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
}
template <int N>
KS_DEV void gload_mat(float* s, const float* g) {
    constexpr int R4 = N / 4;
    for (int q = lane_id(); q < N * R4; q += 32) cp16(s + (q / R4) * TD<N>::P + (q % R4) * 4, g + q * 4);
}
template <int N>
KS_DEV void gload_vec(float* s, const float* g) {
    if (lane_id() < N / 4) cp16(s + lane_id() * 4, g + lane_id() * 4);
}
template <int N>
KS_DEV void gstore_mat(float* g, const float* s) {
    constexpr int R4 = N / 4;
    for (int q = lane_id(); q < N * R4; q += 32)
        *reinterpret_cast<float4*>(g + q * 4) =
            *reinterpret_cast<const float4*>(s + (q / R4) * TD<N>::P + (q % R4) * 4);
}
template <int N>
KS_DEV void gstore_vec(float* g, const float* s) {
    if (lane_id() < N / 4)
        *reinterpret_cast<float4*>(g + lane_id() * 4) = *reinterpret_cast<const float4*>(s + lane_id() * 4);
}

// Global element records: filtering A, C, J, b, eta; smoothing E, L, g.
template <int N>
struct Rec {
    static constexpr int F = 3 * N * N + 2 * N;
    static constexpr int S = 2 * N * N + N;
};
template <int N>
KS_DEV FE gload_fe(const float* g, Pool<N>& pool, Flags& bad) {
    FE e{pool.get(bad), pool.get(bad), pool.get(bad)};
    gload_mat<N>(e.A, g);
    gload_mat<N>(e.C, g + N * N);
    gload_mat<N>(e.J, g + 2 * N * N);
    gload_vec<N>(vrow<N>(e.C), g + 3 * N * N);
    gload_vec<N>(vrow<N>(e.J), g + 3 * N * N + N);
    cp_wait();
    return e;
}
template <int N>
KS_DEV void gstore_fe(float* g, const FE& e) {
    gstore_mat<N>(g, e.A);
    gstore_mat<N>(g + N * N, e.C);
    gstore_mat<N>(g + 2 * N * N, e.J);
    gstore_vec<N>(g + 3 * N * N, vrow<N>(e.C));
    gstore_vec<N>(g + 3 * N * N + N, vrow<N>(e.J));
}
// A filtering prefix state is (b, C) (its A is zero): C and b of a record.
template <int N>
KS_DEV void gload_fstate(float* C, const float* g) {
    gload_mat<N>(C, g + N * N);
    gload_vec<N>(vrow<N>(C), g + 3 * N * N);
    cp_wait();
}
template <int N>
KS_DEV void gstore_fstate(float* g, const float* C) {
    gstore_mat<N>(g + N * N, C);
    gstore_vec<N>(g + 3 * N * N, vrow<N>(C));
}
template <int N>
KS_DEV SE gload_se(const float* g, Pool<N>& pool, Flags& bad) {
    SE e{pool.get(bad), pool.get(bad)};
    gload_mat<N>(e.E, g);
    gload_mat<N>(e.L, g + N * N);
    gload_vec<N>(vrow<N>(e.L), g + 2 * N * N);
    cp_wait();
    return e;
}
template <int N>
KS_DEV void gstore_se(float* g, const SE& e) {
    gstore_mat<N>(g, e.E);
    gstore_mat<N>(g + N * N, e.L);
    gstore_vec<N>(g + 2 * N * N, vrow<N>(e.L));
}
// A smoothing suffix state is (g, L) (its E is zero).
template <int N>
KS_DEV void gload_sstate(float* L, const float* g) {
    gload_mat<N>(L, g + N * N);
    gload_vec<N>(vrow<N>(L), g + 2 * N * N);
    cp_wait();
}
template <int N>
KS_DEV void gstore_sstate(float* g, const float* L) {
    gstore_mat<N>(g + N * N, L);
    gstore_vec<N>(g + 2 * N * N, vrow<N>(L));
}

// ---------------------------------------------------------------- inverse
// Scratch of one warp: vectors (P floats each), the pivot order and a double
// buffer for the pivot row.
template <int N>
struct VS {
    float* p;
    KS_DEV float* v(int i) const { return p + i * TD<N>::P; }
    KS_DEV float* g() const { return p + 3 * TD<N>::P; }                 // up to 2 P floats
    KS_DEV int* piv() const { return reinterpret_cast<int*>(p + 5 * TD<N>::P); }
    KS_DEV float* prow() const { return p + 6 * TD<N>::P; }               // 2 N floats
    static constexpr int FLOATS = 8 * TD<N>::P;
    static_assert(6 * TD<N>::P + 2 * N <= FLOATS, "scratch layout");
};

// out = Mx^{-1} (out distinct from Mx).  Gauss-Jordan with partial pivoting,
// in place: lane l holds row l of Mx^T (column l of Mx, so the loads and the
// final stores are conflict free); at step k the pivot row p_k is the unused
// row with the largest |entry| in column k (one warp max-reduction over
// |entry| with its low 5 mantissa bits replaced by the lane, so ties and
// near-ties go to the lowest lane), the pivot row is broadcast through shared
// memory, and storage column k changes from column k of the matrix to column
// p_k of the inverse of Mx^T.  Then (Mx^T)^{-1}[a][b] = W[p_a][q] with
// p_q = b, i.e. out[p_q][pos(l)] = W[l][q] where pos(l) is the step at which
// lane l was the pivot.
// The steps run in blocks of GJ_U inside a rolled loop: after each block the
// register row is rotated left by GJ_U, so the pivot column of step kb + u is
// always register u (a compile-time index) and the code stays small enough
// for the instruction cache; after N steps the rotation is back to the start.
// PIVOT = false (symmetric positive definite Mx, whose Gauss-Jordan pivots
// stay positive without row exchanges): p_k = k, no search and no final
// permutation.
// Returns the 1-norm condition estimate ||Mx||_1 ||Mx^{-1}||_1 (column sums
// from the registers); `ok` is cleared on a zero or non-finite pivot.
constexpr int GJ_U = 4;

template <int N, bool PIVOT = true>
KS_DEV float gj_inverse(const float* Mx, float* out, VS<N> vs, bool& ok) {
    constexpr int P = TD<N>::P;
    static_assert(N % GJ_U == 0 && GJ_U % 2 == 0, "block of steps");
    const int l = lane_id();
    int* piv = vs.piv();
    float w[N];
#pragma unroll
    for (int c = 0; c < N; ++c) w[c] = Mx[c * P + l];
    float cm = 0.f;
#pragma unroll
    for (int c = 0; c < N; ++c) cm += fabsf(w[c]);
    bool used = false;
    int pos = 0;
    float scale = 1.f;
#pragma unroll 1
    for (int kb = 0; kb < N; kb += GJ_U) {
#pragma unroll
        for (int u = 0; u < GJ_U; ++u) {
            float* pr = vs.prow() + (u & 1) * N;
            int p = kb + u;
            if constexpr (PIVOT) {
                const uint32_t key = used ? 0u : ((__float_as_uint(fabsf(w[u])) & ~31u) | (uint32_t)(31 - l));
                const uint32_t kmax = __reduce_max_sync(kFull, key);
                p = 31 - (int)(kmax & 31u);
            }
            const bool me = (l == p);
            if (me) {
                used = true;
                pos = kb + u;
                piv[kb + u] = p;
#pragma unroll
                for (int j = 0; j < N; j += 4)
                    *reinterpret_cast<float4*>(pr + j) = make_float4(w[j], w[j + 1], w[j + 2], w[j + 3]);
            }
            __syncwarp();
            float rp[N];
#pragma unroll
            for (int j = 0; j < N; j += 4) {
                const float4 t = *reinterpret_cast<const float4*>(pr + j);
                rp[j] = t.x;
                rp[j + 1] = t.y;
                rp[j + 2] = t.z;
                rp[j + 3] = t.w;
            }
            const float pv = rp[u];
            ok = ok && (fabsf(pv) > 1e-30f) && (fabsf(pv) < 3.0e38f);
            const float ip = __frcp_rn(pv);
            // rows are kept unscaled: the true row is scale * w, and a lane
            // takes its scale 1 / pivot when it becomes the pivot row, whose
            // stored values then stay as they are; the update w -= (f / pivot)
            // * pivot row is the same for scaled and unscaled rows.
            const float fp = me ? 0.f : w[u] * ip;
            if (me) scale = ip;
#pragma unroll
            for (int j = 0; j < N; ++j) {
                if (j == u) continue;
                w[j] = fmaf(-fp, rp[j], w[j]);
            }
            w[u] = me ? 1.f : -fp;
        }
        float t[GJ_U];
#pragma unroll
        for (int u = 0; u < GJ_U; ++u) t[u] = w[u];
#pragma unroll
        for (int j = 0; j < N - GJ_U; ++j) w[j] = w[j + GJ_U];
#pragma unroll
        for (int u = 0; u < GJ_U; ++u) w[N - GJ_U + u] = t[u];
    }
    float ci = 0.f;                         // column pos(l) of the inverse
#pragma unroll
    for (int c = 0; c < N; ++c) {
        w[c] *= scale;
        ci += fabsf(w[c]);
    }
    __syncwarp();
    if constexpr (PIVOT) {
#pragma unroll
        for (int q = 0; q < N; q += 4) {
            const int4 pq = *reinterpret_cast<const int4*>(piv + q);
            out[pq.x * P + pos] = w[q];
            out[pq.y * P + pos] = w[q + 1];
            out[pq.z * P + pos] = w[q + 2];
            out[pq.w * P + pos] = w[q + 3];
        }
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) out[q * P + l] = w[q];
    }
    __syncwarp();
    const float nm = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(cm)));
    const float ni = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(ci)));
    return nm * ni;
}

// One step of refinement: lane l forms column l of R = I - Mx X in FP64, then
// X[:, l] += X R[:, l].
template <int N>
KS_DEV void refine_inverse(const float* Mx, float* X) {
    constexpr int P = TD<N>::P;
    const int l = lane_id();
    float rc[N];
    {
        double xc[N];
#pragma unroll
        for (int k = 0; k < N; ++k) xc[k] = (double)X[k * P + l];
#pragma unroll 1
        for (int r = 0; r < N; ++r) {
            double acc = (r == l) ? 1.0 : 0.0;
#pragma unroll
            for (int k = 0; k < N; ++k) acc = fma(-(double)Mx[r * P + k], xc[k], acc);
#pragma unroll
            for (int q = 0; q < N; ++q)
                if (q == r) rc[q] = (float)acc;
        }
    }
    float nc[N];
#pragma unroll 1
    for (int r = 0; r < N; ++r) {
        float s = X[r * P + l];
#pragma unroll
        for (int k = 0; k < N; ++k) s = fmaf(X[r * P + k], rc[k], s);
#pragma unroll
        for (int q = 0; q < N; ++q)
            if (q == r) nc[q] = s;
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < N; ++r) X[r * P + l] = nc[r];
    __syncwarp();
}

// X = Mx^{-1}, refined once when the condition estimate exceeds kRefineCond.
// Returns FL_BAD on a zero or non-finite pivot (then nothing is refined),
// FL_REFINED when the refinement step ran, else 0.
// SPD: Mx is symmetric positive definite (no pivot search).
template <int N, bool SPD = false>
KS_DEV Flags inverse(const float* Mx, float* X, VS<N> vs) {
    bool ok = true;
    const float cond = gj_inverse<N, !SPD>(Mx, X, vs, ok);
    if (!ok) return FL_BAD;
    if (cond > kRefineCond && cond < 3.0e38f) {   // warp-uniform
        refine_inverse<N>(Mx, X);
        return FL_REFINED;
    }
    return 0u;
}

// ---------------------------------------------------------------- model constants
// Filter constants (Lemma 3), padded: A = (I - K H) F, C = Q - K S K^T,
// U = L_S^{-1} H F (ny rows); and the vectors of the measurement elements.
template <int N, int M>
struct alignas(16) FConst {
    float A[N * TD<N>::P];
    float C[N * TD<N>::P];
    float U[M * TD<N>::P];
    float u[N], Kt[M * N], Lsi[M * M], hud[M], b1[N];   // Kt: K transposed
};
// Smoother constants (Lemma 5): F, Q, u.
template <int N, int M>
struct alignas(16) SConst {
    float F[N * TD<N>::P];
    float Q[N * TD<N>::P];
    float u[N];
};

template <int N, int M>
KS_DEV void build_fconst(const ModelConst<N, M>& g, FConst<N, M>& c) {
    constexpr int P = TD<N>::P;
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int a = e / N, b = e % N;
        c.A[a * P + b] = g.A[e];
        c.C[a * P + b] = g.C[sidx(a, b)];
    }
    for (int e = threadIdx.x; e < M * N; e += blockDim.x) c.U[(e / N) * P + e % N] = g.U[e];
    for (int e = threadIdx.x; e < N; e += blockDim.x) {
        c.u[e] = g.u[e];
        c.b1[e] = g.b1[e];
    }
    for (int e = threadIdx.x; e < N * M; e += blockDim.x) c.Kt[(e % M) * N + e / M] = g.K[e];
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) c.Lsi[e] = g.Lsi[e];
    for (int e = threadIdx.x; e < M; e += blockDim.x) c.hud[e] = g.hud[e];
}
template <int N, int M>
KS_DEV void build_sconst(const ModelConst<N, M>& g, SConst<N, M>& c) {
    constexpr int P = TD<N>::P;
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int a = e / N, b = e % N;
        c.F[a * P + b] = g.F[e];
        c.Q[a * P + b] = g.Q[sidx(a, b)];
    }
    for (int e = threadIdx.x; e < N; e += blockDim.x) c.u[e] = g.u[e];
}

// ---------------------------------------------------------------- Lemma 3
// Measurement element k > 1: e = y_k - H u - d, w = L_S^{-1} e (every lane),
// b = u + K e (lane r: row r).
template <int N, int M>
KS_DEV float meas(const FConst<N, M>& c, const float* __restrict__ yk, float (&w)[M]) {
    const int r = lane_id();
    float e[M];
#pragma unroll
    for (int q = 0; q < M; ++q) e[q] = __ldg(yk + q) - c.hud[q];
#pragma unroll
    for (int q = 0; q < M; ++q) {
        float t = 0.f;
#pragma unroll
        for (int p = 0; p <= q; ++p) t = fmaf(c.Lsi[q * M + p], e[p], t);
        w[q] = t;
    }
    float b = c.u[r];
#pragma unroll
    for (int q = 0; q < M; ++q) b = fmaf(c.Kt[q * N + r], e[q], b);
    return b;
}

// The measurement element in full form: A, C constant, J = U^T U, eta = U^T w.
template <int N, int M>
KS_DEV void expand_meas(const FConst<N, M>& c, float b, const float (&w)[M], const FE& o) {
    const int r = lane_id();
    copy_mat<N>(o.A, c.A);
    copy_mat<N>(o.C, c.C);
    mm<N, N, M, TD<N>::P, true, false>(c.U, c.U, o.J);
    float e = 0.f;
#pragma unroll
    for (int q = 0; q < M; ++q) e = fmaf(c.U[q * TD<N>::P + r], w[q], e);
    vrow<N>(o.J)[r] = e;
    vrow<N>(o.C)[r] = b;
    __syncwarp();
}

// The k = 1 element (built in FP64 by the model preparation): A_1 = 0,
// (b_1, C_1), eta_1 = 0, J_1 = 0.  A or J may be null (prefix state only).
template <int N, int M>
KS_DEV void first_elem(const ModelConst<N, M>& g, const FConst<N, M>& c, const FE& o) {
    constexpr int P = TD<N>::P;
    const int r = lane_id();
#pragma unroll 8
    for (int q = 0; q < N; ++q) {
        o.C[q * P + r] = g.C1[sidx(q, r)];
        if (o.A) o.A[q * P + r] = 0.f;
        if (o.J) o.J[q * P + r] = 0.f;
    }
    vrow<N>(o.C)[r] = c.b1[r];
    if (o.J) vrow<N>(o.J)[r] = 0.f;
    __syncwarp();
}

// ---------------------------------------------------------------- Lemma 4
// acc <- acc (x) a_k for the measurement element a_k of Lemma 3 in its
// rank-ny form (J_k = U^T U, eta_k = U^T w).  With G = I + U C U^T = L L^T,
// CUL = C U^T L^{-T} and UL = L^{-1} U, (I + C J_k)^{-1} = I - CUL UL, and
//   X = A (I + C J_k)^{-1} = A - (A CUL) UL,   b <- X (b + C U^T w) + b_k,
//   C <- A (C - CUL CUL^T) A^T + C_k,   A <- X A_acc,
//   eta <- (UL A_acc)^T L^{-1} (w - U b) + eta,   J <- (UL A_acc)^T (UL A_acc) + J.
// PREFIX: acc is a prefix state (A = 0): only b and C are formed.
template <int N, int M, bool PREFIX>
KS_DEV void fcomb_meas(FE& acc, const FConst<N, M>& c, float bk, const float (&w)[M], Pool<N>& pool, VS<N> vs,
                       Flags& bad) {
    constexpr int P = TD<N>::P;
    static_assert(4 * M <= P, "thin products share one buffer");
    const int r = lane_id();
    float* th = pool.get(bad);
    float *CU = th, *CUL = th + M, *ULt = th + 2 * M, *AC = th + 3 * M, *VAt = th;
    float* b = vrow<N>(acc.C);
    mm<N, M, N, P, false, true>(acc.C, c.U, CU);                     // CU = C U^T
    float* G = vs.g();                                               // G = I + U CU
    for (int e = r; e < M * M; e += 32) {
        const int q = e / M, p = e % M;
        float t = (q == p) ? 1.f : 0.f;
#pragma unroll 8
        for (int a = 0; a < N; ++a) t = fmaf(c.U[q * P + a], CU[a * P + p], t);
        G[e] = t;
    }
    __syncwarp();
    float Gp[sym_size(M)];
#pragma unroll
    for (int q = 0; q < M; ++q)
#pragma unroll
        for (int p = 0; p <= q; ++p) Gp[sidx(q, p)] = G[q * M + p];
    float Li[M][M];
    bad |= !chol_inv_lower<M>(Gp, Li);
    {
        float cu[M];
#pragma unroll
        for (int q = 0; q < M; ++q) cu[q] = CU[r * P + q];
        float t = b[r];
#pragma unroll
        for (int q = 0; q < M; ++q) t = fmaf(cu[q], w[q], t);
        vs.v(0)[r] = t;                                              // t = b + C U^T w
#pragma unroll
        for (int q = 0; q < M; ++q) {
            float s = 0.f, u = 0.f;
#pragma unroll
            for (int p = 0; p <= q; ++p) {
                s = fmaf(cu[p], Li[q][p], s);
                u = fmaf(Li[q][p], c.U[p * P + r], u);
            }
            CUL[r * P + q] = s;
            ULt[r * P + q] = u;
        }
        if constexpr (!PREFIX) {
            float wr = 0.f;
#pragma unroll
            for (int q = 0; q < M; ++q)
                if (q == r) wr = w[q];
            if (r < M) vs.v(1)[r] = wr - rdot<N>(c.U, r, b);          // w - U b (lane q < M)
        }
    }
    __syncwarp();
    mm<N, M, N, P, false, false>(c.A, CUL, AC);                       // A CUL
    float* X = pool.get(bad);
    mm<N, N, M, P, false, true>(AC, ULt, X, c.A, -1.f);              // X = A - (A CUL) UL
    b[r] = rdot<N>(X, r, vs.v(0)) + bk;
    if constexpr (!PREFIX) {
        float* An = pool.get(bad);
        mmq<N, false, false>(X, acc.A, An);                           // A <- X A
        mm<N, M, N, P, true, false>(acc.A, ULt, VAt);                 // VAt = A^T UL^T
        pool.put(acc.A);
        acc.A = An;
        float sv[M];                                                  // L^{-1} (w - U b)
#pragma unroll
        for (int q = 0; q < M; ++q) {
            float t = 0.f;
#pragma unroll
            for (int p = 0; p <= q; ++p) t = fmaf(Li[q][p], vs.v(1)[p], t);
            sv[q] = t;
        }
        float e = vrow<N>(acc.J)[r];
#pragma unroll
        for (int q = 0; q < M; ++q) e = fmaf(VAt[r * P + q], sv[q], e);
        vrow<N>(acc.J)[r] = e;
        mm<N, N, M, P, false, true>(VAt, VAt, acc.J, acc.J);          // J <- VA^T VA + J
    }
    mm<N, N, M, P, false, true>(CUL, CUL, acc.C, acc.C, -1.f);        // W = C - CUL CUL^T
    mmq<N, false, true>(c.A, acc.C, X);                               // Y = A W  (W symmetric)
    mmq<N, false, true>(X, c.A, acc.C, c.C);                          // C <- Y A^T + C_k
    symm<N>(acc.C);
    pool.put(X);
    pool.put(th);
}

// st <- st (x) j for a prefix state st = (b, C) (A = 0): only b and C.
//   M = I + C J_j,  X = A_j M^{-1},  b <- X (b + C eta_j) + b_j,  C <- X C A_j^T + C_j.
template <int N>
KS_DEV void fadvance(FE& st, const FE& j, Pool<N>& pool, VS<N> vs, Flags& bad) {
    const int r = lane_id();
    float* s0 = pool.get(bad);
    float* s1 = pool.get(bad);
    mmq<N, false, true>(st.C, j.J, s0);
    add_diag<N>(s0, 1.f);
    vs.v(0)[r] = vrow<N>(st.C)[r] + rdot<N>(st.C, r, vrow<N>(j.J));
    bad |= inverse<N>(s0, s1, vs);
    mmq<N, false, false>(j.A, s1, s0);                                // X = A_j M^{-1}
    mmq<N, false, true>(s0, st.C, s1);                                // X C
    vrow<N>(st.C)[r] = rdot<N>(s0, r, vs.v(0)) + vrow<N>(j.C)[r];
    mmq<N, false, true>(s1, j.A, st.C, j.C);                          // X C A_j^T + C_j
    symm<N>(st.C);
    pool.put(s0);
    pool.put(s1);
}

// o = i (x) j (general Lemma 4 operator); i and j are left intact.
//   M = I + C_i J_j,  X = A_j M^{-1},  A_o = X A_i,  b_o = X (b_i + C_i eta_j) + b_j,
//   C_o = X C_i A_j^T + C_j,  eta_o = A_i^T M^{-T} (eta_j - J_j b_i) + eta_i,
//   J_o = A_i^T (M^{-T} J_j) A_i + J_i.
template <int N>
KS_DEV FE fcombine(const FE& i, const FE& j, Pool<N>& pool, VS<N> vs, Flags& bad) {
    const int r = lane_id();
    float* s0 = pool.get(bad);
    mmq<N, false, true>(i.C, j.J, s0);
    add_diag<N>(s0, 1.f);
    vs.v(0)[r] = vrow<N>(i.C)[r] + rdot<N>(i.C, r, vrow<N>(j.J));    // t = b_i + C_i eta_j
    vs.v(1)[r] = vrow<N>(j.J)[r] - rdot<N>(j.J, r, vrow<N>(i.C));    // v = eta_j - J_j b_i
    float* s1 = pool.get(bad);
    bad |= inverse<N>(s0, s1, vs);                             // M^{-1}
    float* s2 = pool.get(bad);
    float* s3 = pool.get(bad);
    mmq<N, false, false>(j.A, s1, s2);                                // X
    mmq<N, true, true>(s1, j.J, s3);                                  // Vm = M^{-T} J_j
    vs.v(2)[r] = cdot<N>(s1, r, vs.v(1));                             // M^{-T} v
    __syncwarp();
    mmq<N, false, true>(s2, i.C, s1);                                 // X C_i
    float* s4 = pool.get(bad);
    mmq<N, false, false>(s2, i.A, s4);                                // A_o
    vrow<N>(s0)[r] = rdot<N>(s2, r, vs.v(0)) + vrow<N>(j.C)[r];      // b_o
    mmq<N, false, true>(s1, j.A, s0, j.C);                            // C_o
    symm<N>(s0);
    mmq<N, false, false>(s3, i.A, s2);                                // Vm A_i
    mmq<N, true, false>(i.A, s2, s1, i.J);                            // J_o
    vrow<N>(s1)[r] = cdot<N>(i.A, r, vs.v(2)) + vrow<N>(i.J)[r];     // eta_o
    symm<N>(s1);
    pool.put(s2);
    pool.put(s3);
    return FE{s4, s0, s1};
}

// ---------------------------------------------------------------- Lemma 5
// Smoothing element from the filtered posterior (xbar, P), given as the buffer
// Pm (P in the rows, xbar in the vector row); Pm is consumed.
//   k < n: P- = F P F^T + Q,  E = P F^T (P-)^{-1},  g = xbar - E (F xbar + u),
//          L = P - E F P;     k = n: (0, xbar, P).
template <int N, int M>
KS_DEV SE selem(float* Pm, const SConst<N, M>& c, bool last, Pool<N>& pool, VS<N> vs, Flags& bad) {
    const int r = lane_id();
    if (last) {
        float* E = pool.get(bad);
        zero_mat<N>(E);
        return SE{E, Pm};
    }
    const float* xb = vrow<N>(Pm);
    float* FP = pool.get(bad);
    mmq<N, false, true>(c.F, Pm, FP);                                 // F P
    float* Pp = pool.get(bad);
    mmq<N, false, true>(FP, c.F, Pp, c.Q);                            // P- = F P F^T + Q
    vs.v(0)[r] = rdot<N>(c.F, r, xb) + c.u[r];                        // F xbar + u
    float* Pi = pool.get(bad);
    bad |= inverse<N, true>(Pp, Pi, vs);                           // P- is SPD
    mmq<N, true, true>(FP, Pi, Pp);                                   // E = (F P)^T (P-)^{-1}
    mmq<N, false, false>(Pp, FP, Pi, Pm, -1.f);                       // L = P - E F P
    vrow<N>(Pi)[r] = xb[r] - rdot<N>(Pp, r, vs.v(0));                 // g
    symm<N>(Pi);
    pool.put(FP);
    pool.put(Pm);
    return SE{Pp, Pi};
}

// ---------------------------------------------------------------- Lemma 6
// o = i (x) j with i the earlier step: E = E_i E_j, g = E_i g_j + g_i,
// L = E_i L_j E_i^T + L_i.  L and g are formed in place in i's buffer (o.L is
// i.L); STATE: j is a suffix state (E_j = 0) and o.E is null; otherwise o.E is
// a fresh buffer.  i.E and j are left for the caller to release.
template <int N, bool STATE>
KS_DEV SE scombine(const SE& i, const SE& j, Pool<N>& pool, Flags& bad) {
    const int r = lane_id();
    float* Y = pool.get(bad);
    mmq<N, false, true>(i.E, j.L, Y);                                 // E_i L_j
    vrow<N>(i.L)[r] += rdot<N>(i.E, r, vrow<N>(j.L));
    mmq<N, false, true>(Y, i.E, i.L, i.L);                            // Y E_i^T + L_i
    symm<N>(i.L);
    pool.put(Y);
    float* En = nullptr;
    if constexpr (!STATE) {
        En = pool.get(bad);
        mmq<N, false, false>(i.E, j.E, En);
    }
    return SE{En, i.L};
}

}  // namespace tc
}  // namespace ks
