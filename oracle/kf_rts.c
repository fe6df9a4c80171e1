/*
 * FP64 sequential Kalman filter and Rauch-Tung-Striebel smoother.
 *
 * TEST INFRASTRUCTURE: this is the oracle that the GPU path is checked
 * against.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it; the product path never does.
 *
 * What it computes is the plain definition of the result the parallel method
 * reaches: Theorem 1 (Section III-A) says that the all-prefix-sums of the
 * filtering elements are the filtering densities p(x_k | y_{1:k}), and
 * Theorem 2 (Section III-B) says that the suffix sums of the smoothing
 * elements are the smoothing densities p(x_k | y_{1:n}).  For the
 * linear/Gaussian model of Section IV these densities are produced exactly by
 * the classic Kalman filter and RTS smoother (Section II-A), which this file
 * writes out step by step with no blocking, fusion or reordering:
 *
 *   filter (the k = 1 equations of Lemma 3 applied at every step k):
 *     m- = F_{k-1} m_{k-1} + u_{k-1}
 *     P- = F_{k-1} P_{k-1} F_{k-1}^T + Q_{k-1}
 *     S  = H_k P- H_k^T + R_k
 *     K  = P- H_k^T S^{-1}
 *     m_k = m- + K (y_k - H_k m- - d_k)
 *     P_k = P- - K S K^T
 *   smoother (Lemma 5's E_k is the RTS gain), for k = n-1 .. 1:
 *     P-_{k+1} = F_k P_k F_k^T + Q_k
 *     G_k  = P_k F_k^T (P-_{k+1})^{-1}
 *     ms_k = m_k + G_k (ms_{k+1} - F_k m_k - u_k)
 *     Ps_k = P_k + G_k (Ps_{k+1} - P-_{k+1}) G_k^T
 *   starting from ms_n = m_n, Ps_n = P_n.
 *
 * Indexing: arrays are 0-based over steps i = k - 1.  Per-step model arrays
 * (time-varying case) are indexed so that entry i holds the parameters used
 * at step i: F[i], u[i], Q[i] move the state from step i-1 to step i (F_{k-1}
 * in Section IV), and H[i], d[i], R[i] measure step i.  The smoother at step i
 * therefore uses F[i+1], u[i+1], Q[i+1].  A stride of 0 means time-invariant.
 *
 * All matrices are dense row-major.  Plain loops, no fast-math.
 * The marginal log-likelihood terms log p(y_k | y_{1:k-1}) (Section III-C)
 * are returned per step when `loglik` is non-NULL.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* C[n x m] = A[n x k] * B[k x m] */
static void mm(const double *A, const double *B, double *C, int n, int k, int m) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * m + j];
            C[i * m + j] = s;
        }
}

/* C[n x m] = A[n x k] * B[m x k]^T */
static void mmt(const double *A, const double *B, double *C, int n, int k, int m) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += A[i * k + l] * B[j * k + l];
            C[i * m + j] = s;
        }
}

/* y[n] = A[n x k] x[k] */
static void mv(const double *A, const double *x, double *y, int n, int k) {
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int l = 0; l < k; ++l) s += A[i * k + l] * x[l];
        y[i] = s;
    }
}

/* Cholesky S = L L^T of an n x n SPD matrix; returns 0 on success. */
static int cholesky(const double *S, double *L, int n) {
    memset(L, 0, sizeof(double) * (size_t)n * n);
    for (int j = 0; j < n; ++j) {
        double s = S[j * n + j];
        for (int l = 0; l < j; ++l) s -= L[j * n + l] * L[j * n + l];
        if (!(s > 0.0)) return -1;
        double ljj = sqrt(s);
        L[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = S[i * n + j];
            for (int l = 0; l < j; ++l) t -= L[i * n + l] * L[j * n + l];
            L[i * n + j] = t / ljj;
        }
    }
    return 0;
}

/* X[n x r] = S^{-1} B[n x r] for SPD S, by Cholesky; returns 0 on success. */
static int spd_solve(const double *S, const double *B, double *X, int n, int r, double *work) {
    double *L = work;
    if (cholesky(S, L, n)) return -1;
    for (int c = 0; c < r; ++c) {
        for (int i = 0; i < n; ++i) {            /* L z = b */
            double t = B[i * r + c];
            for (int l = 0; l < i; ++l) t -= L[i * n + l] * X[l * r + c];
            X[i * r + c] = t / L[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {       /* L^T x = z */
            double t = X[i * r + c];
            for (int l = i + 1; l < n; ++l) t -= L[l * n + i] * X[l * r + c];
            X[i * r + c] = t / L[i * n + i];
        }
    }
    return 0;
}

/* log det of SPD S via Cholesky (work holds L from the last spd_solve). */
static double logdet_from_chol(const double *L, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += log(L[i * n + i]);
    return 2.0 * s;
}

/*
 * Sequential Kalman filter.  Strides sF.. are the per-step strides of the
 * model arrays in doubles (0 for a time-invariant model).
 * Returns 0, or -(i+1) if the innovation covariance at step i is not SPD.
 */
int oracle_kf(int nx, int ny, int64_t T,
              const double *F, int64_t sF, const double *u, int64_t su,
              const double *Q, int64_t sQ, const double *H, int64_t sH,
              const double *d, int64_t sd, const double *R, int64_t sR,
              const double *m0, const double *P0, const double *y,
              double *fmean, double *fcov, double *loglik) {
    const int n = nx, m = ny;
    const int w = n > m ? n : m;
    double *buf = (double *)calloc((size_t)(6 * n * n + 4 * n * m + 3 * m * m + 3 * n + 2 * m + w * w), sizeof(double));
    if (!buf) return -1000000;
    double *mp = buf;              /* m-          [n]     */
    double *Pp = mp + n;           /* P-          [n x n] */
    double *FP = Pp + n * n;       /* F P         [n x n] */
    double *HP = FP + n * n;       /* H P-        [m x n] */
    double *S = HP + m * n;        /* S           [m x m] */
    double *KT = S + m * m;        /* K^T         [m x n] */
    double *K = KT + m * n;        /* K           [n x m] */
    double *KS = K + n * m;        /* K S         [n x m] */
    double *KSK = KS + n * m;      /* K S K^T     [n x n] */
    double *mprev = KSK + n * n;   /* [n] */
    double *Pprev = mprev + n;     /* [n x n] */
    double *e = Pprev + n * n;     /* innovation  [m] */
    double *Se = e + m;            /* S^{-1} e    [m] */
    double *work = Se + m;         /* Cholesky factor [w x w] */
    memcpy(mprev, m0, sizeof(double) * n);
    memcpy(Pprev, P0, sizeof(double) * n * n);
    int rc = 0;
    for (int64_t i = 0; i < T; ++i) {
        const double *Fi = F + i * sF, *ui = u + i * su, *Qi = Q + i * sQ;
        const double *Hi = H + i * sH, *di = d + i * sd, *Ri = R + i * sR;
        /* predict */
        mv(Fi, mprev, mp, n, n);
        for (int a = 0; a < n; ++a) mp[a] += ui[a];
        mm(Fi, Pprev, FP, n, n, n);
        mmt(FP, Fi, Pp, n, n, n);
        for (int a = 0; a < n * n; ++a) Pp[a] += Qi[a];
        /* update */
        mm(Hi, Pp, HP, m, n, n);                 /* H P-        [m x n] */
        mmt(HP, Hi, S, m, n, m);                 /* H P- H^T    [m x m] */
        for (int a = 0; a < m * m; ++a) S[a] += Ri[a];
        if (spd_solve(S, HP, KT, m, n, work)) { rc = -(int)(i + 1); break; }  /* K^T = S^{-1} H P- */
        mv(Hi, mp, e, m, n);
        for (int a = 0; a < m; ++a) e[a] = y[i * m + a] - e[a] - di[a];
        double *mk = fmean + i * n, *Pk = fcov + i * n * n;
        for (int a = 0; a < n; ++a) {            /* m = m- + K e */
            double s = 0.0;
            for (int b = 0; b < m; ++b) s += KT[b * n + a] * e[b];
            mk[a] = mp[a] + s;
        }
        /* P = P- - K S K^T */
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < m; ++b) K[a * m + b] = KT[b * n + a];
        mm(K, S, KS, n, m, m);
        mmt(KS, K, KSK, n, m, n);
        for (int a = 0; a < n * n; ++a) Pk[a] = Pp[a] - KSK[a];
        if (loglik) {
            /* log N(y_k; H m- + d, S): S^{-1} e through the Cholesky factor */
            if (spd_solve(S, e, Se, m, 1, work)) { rc = -(int)(i + 1); break; }
            double q = 0.0;
            for (int a = 0; a < m; ++a) q += e[a] * Se[a];
            loglik[i] = -0.5 * (q + logdet_from_chol(work, m) + m * 1.8378770664093454835606594728112 /* log(2 pi) */);
        }
        memcpy(mprev, mk, sizeof(double) * n);
        memcpy(Pprev, Pk, sizeof(double) * n * n);
    }
    free(buf);
    return rc;
}

/*
 * RTS smoother from filtered means/covariances.  Returns 0, or -(i+1) if the
 * predicted covariance at step i+1 is not SPD.
 */
int oracle_rts(int nx, int64_t T, const double *F, int64_t sF, const double *u, int64_t su,
               const double *Q, int64_t sQ, const double *fmean, const double *fcov,
               double *smean, double *scov) {
    const int n = nx;
    if (T <= 0) return 0;
    double *buf = (double *)calloc((size_t)(8 * n * n + 4 * n), sizeof(double));
    if (!buf) return -1000000;
    double *FP = buf, *Pp = FP + n * n, *GT = Pp + n * n, *D = GT + n * n, *tmp = D + n * n;
    double *work = tmp + n * n, *r = work + n * n, *Fm = r + n;
    memcpy(smean + (T - 1) * n, fmean + (T - 1) * n, sizeof(double) * n);
    memcpy(scov + (T - 1) * n * n, fcov + (T - 1) * n * n, sizeof(double) * n * n);
    int rc = 0;
    for (int64_t i = T - 2; i >= 0; --i) {
        const double *Fk = F + (i + 1) * sF, *uk = u + (i + 1) * su, *Qk = Q + (i + 1) * sQ;
        const double *mk = fmean + i * n, *Pk = fcov + i * n * n;
        mm(Fk, Pk, FP, n, n, n);                 /* F P */
        mmt(FP, Fk, Pp, n, n, n);                /* F P F^T */
        for (int a = 0; a < n * n; ++a) Pp[a] += Qk[a];
        if (spd_solve(Pp, FP, GT, n, n, work)) { rc = -(int)(i + 2); break; }  /* G^T = (P-)^{-1} F P */
        mv(Fk, mk, Fm, n, n);
        for (int a = 0; a < n; ++a) r[a] = smean[(i + 1) * n + a] - Fm[a] - uk[a];
        for (int a = 0; a < n; ++a) {
            double s = 0.0;
            for (int b = 0; b < n; ++b) s += GT[b * n + a] * r[b];
            smean[i * n + a] = mk[a] + s;
        }
        for (int a = 0; a < n * n; ++a) D[a] = scov[(i + 1) * n * n + a] - Pp[a];
        /* tmp = G D = GT^T D ; Ps = P + tmp G^T */
        for (int a = 0; a < n; ++a)
            for (int c = 0; c < n; ++c) {
                double s = 0.0;
                for (int b = 0; b < n; ++b) s += GT[b * n + a] * D[b * n + c];
                tmp[a * n + c] = s;
            }
        for (int a = 0; a < n; ++a)
            for (int c = 0; c < n; ++c) {
                double s = 0.0;
                for (int b = 0; b < n; ++b) s += tmp[a * n + b] * GT[b * n + c];
                scov[i * n * n + a * n + c] = Pk[a * n + c] + s;
            }
    }
    free(buf);
    return rc;
}

/* Filter followed by smoother. */
int oracle_kf_rts(int nx, int ny, int64_t T,
                  const double *F, int64_t sF, const double *u, int64_t su,
                  const double *Q, int64_t sQ, const double *H, int64_t sH,
                  const double *d, int64_t sd, const double *R, int64_t sR,
                  const double *m0, const double *P0, const double *y,
                  double *fmean, double *fcov, double *smean, double *scov, double *loglik) {
    int rc = oracle_kf(nx, ny, T, F, sF, u, su, Q, sQ, H, sH, d, sd, R, sR, m0, P0, y,
                       fmean, fcov, loglik);
    if (rc) return rc;
    return oracle_rts(nx, T, F, sF, u, su, Q, sQ, fmean, fcov, smean, scov);
}
