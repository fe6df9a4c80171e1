// ks_loglik.cu -- marginal log-likelihood by one extra parallel pass over the
// filtered moments (Section III-C: Theorem 1's prefix also carries p(y_1:k)).
//
// p(y_1:n) = prod_k p(y_k | y_1:k-1) and, for the linear/Gaussian model,
//   p(y_k | y_1:k-1) = N(y_k; mu_k, S_k),  mu_k = G xbar_{k-1} + c0,
//   S_k = G P_{k-1} G^T + S0,  G = H F,  S0 = H Q H^T + R,  c0 = H u + d,
// with (xbar_{k-1}, P_{k-1}) the filtered posterior of the previous step and
// (m0, P0) in place of it at k = 1.  One thread per step forms S_k, its
// Cholesky factor, the quadratic form and log det S_k; the per-step values
// are written in FP32 and summed in FP64 (block sums, one atomic per block).
#include <cuda_runtime.h>

#include "../../include/ks.h"

namespace ks {
namespace {

constexpr int kLLThreads = 128;
constexpr double kLog2Pi = 1.8378770664093453;

template <int N, int M>
struct LLConst {
    float G[M * N];      // H F
    float S0[M * M];     // H Q H^T + R
    float c0[M];         // H u + d
};

template <int N, int M>
__device__ void build_llconst(const float* __restrict__ F, const float* __restrict__ u, const float* __restrict__ Q,
                              const float* __restrict__ H, const float* __restrict__ d, const float* __restrict__ R,
                              LLConst<N, M>& c, float* HQ) {
    const int t = threadIdx.x, nt = blockDim.x;
    for (int e = t; e < M * N; e += nt) {
        const int q = e / N, a = e % N;
        float g = 0.f, h = 0.f;
        for (int k = 0; k < N; ++k) {
            g = fmaf(H[q * N + k], F[k * N + a], g);
            h = fmaf(H[q * N + k], Q[k * N + a], h);
        }
        c.G[e] = g;
        HQ[e] = h;
    }
    for (int q = t; q < M; q += nt) {
        float s = d ? d[q] : 0.f;
        if (u)
            for (int k = 0; k < N; ++k) s = fmaf(H[q * N + k], u[k], s);
        c.c0[q] = s;
    }
    __syncthreads();
    for (int e = t; e < M * M; e += nt) {
        const int q = e / M, p = e % M;
        float s = 0.5f * (R[q * M + p] + R[p * M + q]);
        for (int k = 0; k < N; ++k) s = fmaf(HQ[q * N + k], H[p * N + k], s);
        c.S0[e] = s;
    }
    __syncthreads();
}

// log N(r; 0, S) for an M x M SPD matrix S (row-major, lower triangle read);
// returns false when the Cholesky factorisation fails.
template <int M, class Real>
__device__ bool log_gauss(Real (&S)[M][M], Real (&r)[M], Real& out) {
    Real ld = 0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        Real s = S[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= S[j][k] * S[j][k];
        if (!(s > Real(0))) return false;
        const Real l = sqrt(s);
        S[j][j] = l;
        ld += log(l);
#pragma unroll
        for (int i = j + 1; i < M; ++i) {
            Real t = S[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= S[i][k] * S[j][k];
            S[i][j] = t / l;
        }
    }
    Real q = 0;                                     // || L^{-1} r ||^2
#pragma unroll
    for (int i = 0; i < M; ++i) {
        Real t = r[i];
#pragma unroll
        for (int k = 0; k < i; ++k) t -= S[i][k] * r[k];
        r[i] = t / S[i][i];
        q += r[i] * r[i];
    }
    out = Real(-0.5) * (q + Real(M) * Real(kLog2Pi)) - ld;
    return true;
}

template <int N, int M>
__global__ void __launch_bounds__(kLLThreads) loglik_kernel(
    const float* __restrict__ F, const float* __restrict__ u, const float* __restrict__ Q,
    const float* __restrict__ H, const float* __restrict__ d, const float* __restrict__ R,
    const double* __restrict__ m0, const double* __restrict__ P0, const float* __restrict__ y, int64_t T,
    const float* __restrict__ fmean, const float* __restrict__ fcov, float* __restrict__ ll,
    double* __restrict__ total, uint32_t* __restrict__ bad_out) {
    __shared__ LLConst<N, M> c;
    __shared__ float HQ[M * N];
    __shared__ double red[kLLThreads / 32];
    build_llconst<N, M>(F, u, Q, H, d, R, c, HQ);
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double val = 0.0;
    bool bad = false;
    if (k == 0) {                                   // from the prior, in FP64
        double S[M][M], r[M];
        for (int q = 0; q < M; ++q) {
            double gm = c.c0[q];
            for (int a = 0; a < N; ++a) gm += (double)c.G[q * N + a] * m0[a];
            r[q] = (double)y[q] - gm;
        }
        for (int q = 0; q < M; ++q) {
            double gp[N];
            for (int b = 0; b < N; ++b) {
                double s = 0.0;
                for (int a = 0; a < N; ++a) s += (double)c.G[q * N + a] * P0[a * N + b];
                gp[b] = s;
            }
            for (int p = 0; p <= q; ++p) {
                double s = c.S0[q * M + p];
                for (int b = 0; b < N; ++b) s += gp[b] * (double)c.G[p * N + b];
                S[q][p] = s;
            }
        }
        double v;
        bad = !log_gauss<M, double>(S, r, v);
        val = v;
    } else if (k < T) {
        const float* xb = fmean + (k - 1) * N;
        const float* P = fcov + (k - 1) * N * N;
        float S[M][M], r[M];
#pragma unroll
        for (int q = 0; q < M; ++q) {
            float gm = c.c0[q];
#pragma unroll 8
            for (int a = 0; a < N; ++a) gm = fmaf(c.G[q * N + a], __ldg(xb + a), gm);
            r[q] = __ldg(y + k * M + q) - gm;
        }
#pragma unroll 1
        for (int q = 0; q < M; ++q) {
            float gp[N];
#pragma unroll
            for (int b = 0; b < N; ++b) gp[b] = 0.f;
#pragma unroll 4
            for (int a = 0; a < N; ++a) {
                const float g = c.G[q * N + a];
#pragma unroll
                for (int b = 0; b < N; ++b) gp[b] = fmaf(g, __ldg(P + a * N + b), gp[b]);
            }
#pragma unroll
            for (int p = 0; p < M; ++p) {
                if (p > q) break;
                float s = c.S0[q * M + p];
#pragma unroll
                for (int b = 0; b < N; ++b) s = fmaf(gp[b], c.G[p * N + b], s);
                S[q][p] = s;
            }
        }
        float v;
        bad = !log_gauss<M, float>(S, r, v);
        val = v;
    }
    if (k < T) {
        if (ll) ll[k] = (float)val;
        bad = bad || !isfinite(val);
    }
    // FP64 block sum, one atomic per block
    for (int off = 16; off > 0; off >>= 1) val += __shfl_down_sync(0xffffffffu, val, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = val;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < kLLThreads / 32; ++i) s += red[i];
        if (total) atomicAdd(total, s);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(bad_out, 1u);
}

template <int N, int M>
int launch(const ks_model* m, const float* y, int64_t T, const float* fm, const float* fc, float* ll, double* total,
           uint32_t* bad, cudaStream_t st) {
    const int64_t blocks = (T + kLLThreads - 1) / kLLThreads;
    loglik_kernel<N, M><<<(unsigned)blocks, kLLThreads, 0, st>>>(m->F, m->u, m->Q, m->H, m->d, m->R, m->m0, m->P0,
                                                                 y, T, fm, fc, ll, total, bad);
    return cudaGetLastError() == cudaSuccess ? KS_OK : KS_ECUDA;
}

}  // namespace
}  // namespace ks

extern "C" int ks_loglik(const ks_model* m, const float* y, int64_t T, const float* fmean, const float* fcov,
                         float* ll, double* total, uint32_t* status, void* stream) {
    using namespace ks;
    if (!m || !m->F || !m->Q || !m->H || !m->R || !m->m0 || !m->P0 || !y) return KS_EINVAL;
    if (m->time_varying != 0) return KS_EUNSUPPORTED;
    if (T < 1 || T > 0x7fffffffLL || (T > 1 && (!fmean || !fcov)) || !status) return KS_EINVAL;
    if (!ll && !total) return KS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (total && cudaMemsetAsync(total, 0, sizeof(double), st) != cudaSuccess) return KS_ECUDA;
    if (cudaMemsetAsync(status, 0, sizeof(uint32_t), st) != cudaSuccess) return KS_ECUDA;
    const int nx = m->nx, ny = m->ny;
    if (nx == 2 && ny == 1) return launch<2, 1>(m, y, T, fmean, fcov, ll, total, status, st);
    if (nx == 4 && ny == 2) return launch<4, 2>(m, y, T, fmean, fcov, ll, total, status, st);
    if (nx == 6 && ny == 3) return launch<6, 3>(m, y, T, fmean, fcov, ll, total, status, st);
    if (nx == 8 && ny == 4) return launch<8, 4>(m, y, T, fmean, fcov, ll, total, status, st);
    if (nx == 32 && ny == 8) return launch<32, 8>(m, y, T, fmean, fcov, ll, total, status, st);
    return KS_EUNSUPPORTED;
}
