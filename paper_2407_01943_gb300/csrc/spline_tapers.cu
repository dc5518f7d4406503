// Nominal tapers without the GEP: interpolated DPSS (Table 1, step 3, case
// f_c0 = 0, sub-steps (a)-(c)).
//
//   (a) DPSS on N uniform nodes u_j = t_1 + j D, D = (t_N - t_1) / (N - 1),
//       half-bandwidth W = f_w D cycles per node.  The sequences are the top
//       eigenvectors of the symmetric tridiagonal matrix that commutes with
//       the prolate matrix (Slepian 1978; Percival & Walden 1993, Sec. 8.3):
//         diag_j = ((N - 1 - 2j) / 2)^2 cos(2 pi W),  offdiag_j = j (N - j) / 2.
//       Its eigenvalues are well separated (unlike the prolate matrix's, which
//       crowd at 1), so each sequence is computed on its own: Sturm-sequence
//       bisection for the eigenvalue, then inverse iteration with a pivoted
//       tridiagonal LU.  O(N) per bisection step and per solve.
//   (b) each sequence is carried to the sampling times by a not-a-knot cubic
//       spline through the nodes (second derivatives from a tridiagonal
//       system; uniform spacing).
//   (c) w_k is scaled to w^T R(B) w = 2 f_w (Eq. bg_norm_requirement).  The
//       quadratic forms w^T R(B) w and w^T R(A0) w are FP64 pair sums on the
//       GPU (no N x N matrix is formed); lambda_k = w^T R(A0) w / w^T R(B) w is
//       the concentration the interpolated taper attains, used by the leakage
//       estimate.
// The caller applies the sign rule shared with the GEP tapers.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace m2 {
namespace {

constexpr double kPiD = 3.141592653589793238462643383279502884;
constexpr int kQuadRows = 32;  // rows n per CTA of the quadratic-form kernel

// Number of eigenvalues of the tridiagonal (d, e) below x (Sturm sequence; e[j] couples j-1 and j).
int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x, double tiny) {
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0) ++cnt;
    for (size_t j = 1; j < d.size(); ++j) {
        if (std::fabs(q) < tiny) q = q < 0 ? -tiny : tiny;
        q = (d[j] - x) - e[j] * e[j] / q;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// Eigenvector of the tridiagonal for eigenvalue lam by inverse iteration: (T - lam I) y = b with
// an LU factorisation with partial pivoting (rows i and i+1 swapped when |sub| > |diag|).
void inverse_iteration(const std::vector<double>& d0, const std::vector<double>& e, double lam, double tiny,
                       std::vector<double>& y) {
    const size_t n = d0.size();
    std::vector<double> d(n), dl(n > 1 ? n - 1 : 1), du(n > 1 ? n - 1 : 1), du2(n > 2 ? n - 2 : 1);
    std::vector<char> swp(n > 1 ? n - 1 : 1, 0);
    for (size_t i = 0; i < n; ++i) d[i] = d0[i] - lam;
    for (size_t i = 0; i + 1 < n; ++i) {
        dl[i] = e[i + 1];
        du[i] = e[i + 1];
    }
    for (size_t i = 0; i + 1 < n; ++i) {
        if (std::fabs(d[i]) >= std::fabs(dl[i])) {
            if (std::fabs(d[i]) < tiny) d[i] = tiny;
            const double f = dl[i] / d[i];
            dl[i] = f;
            d[i + 1] -= f * du[i];
            if (i + 2 < n) du2[i] = 0.0;
            swp[i] = 0;
        } else {
            const double f = d[i] / dl[i];
            d[i] = dl[i];
            dl[i] = f;
            const double t = du[i];
            du[i] = d[i + 1];
            d[i + 1] = t - f * d[i + 1];
            if (i + 2 < n) {
                du2[i] = du[i + 1];
                du[i + 1] = -f * du[i + 1];
            }
            swp[i] = 1;
        }
    }
    if (std::fabs(d[n - 1]) < tiny) d[n - 1] = tiny;
    // start vector: deterministic, not orthogonal to any eigenvector in practice
    y.assign(n, 0.0);
    for (size_t i = 0; i < n; ++i) y[i] = 1.0 + 0.5 * std::sin(0.7 * (double)i + 0.3);
    for (int it = 0; it < 3; ++it) {
        // forward: L
        for (size_t i = 0; i + 1 < n; ++i) {
            if (!swp[i]) {
                y[i + 1] -= dl[i] * y[i];
            } else {
                const double t = y[i];
                y[i] = y[i + 1];
                y[i + 1] = t - dl[i] * y[i];
            }
        }
        // back: U (diag d, super du, second super du2)
        y[n - 1] /= d[n - 1];
        if (n >= 2) y[n - 2] = (y[n - 2] - du[n - 2] * y[n - 1]) / d[n - 2];
        for (size_t ii = n >= 3 ? n - 3 + 1 : 0; ii-- > 0;) y[ii] = (y[ii] - du[ii] * y[ii + 1] - du2[ii] * y[ii + 2]) / d[ii];
        double nrm = 0;
        for (double v : y) nrm += v * v;
        nrm = std::sqrt(nrm);
        for (double& v : y) v /= nrm;
    }
}

// The K leading DPSS (unit norm) of length N, half-bandwidth W (cycles per node), [K][N].
void dpss_tridiagonal(int N, double W, int K, std::vector<double>& v) {
    std::vector<double> d(N), e(N, 0.0);
    const double cw = std::cos(2.0 * kPiD * W);
    for (int j = 0; j < N; ++j) {
        const double a = 0.5 * (double)(N - 1 - 2 * j);
        d[j] = a * a * cw;
    }
    for (int j = 1; j < N; ++j) e[j] = 0.5 * (double)j * (double)(N - j);
    double lo = d[0], hi = d[0];
    for (int j = 0; j < N; ++j) {
        const double r = (j > 0 ? std::fabs(e[j]) : 0.0) + (j + 1 < N ? std::fabs(e[j + 1]) : 0.0);
        lo = std::min(lo, d[j] - r);
        hi = std::max(hi, d[j] + r);
    }
    const double scale = std::max(std::fabs(lo), std::fabs(hi));
    const double tiny = 1e-300 + scale * 1e-300;
    v.assign((size_t)K * N, 0.0);
    std::vector<double> y;
    for (int k = 0; k < K; ++k) {
        const int idx = N - 1 - k;  // ascending index of the k-th largest eigenvalue
        double a = lo, b = hi;      // count(a) <= idx < count(b)
        for (int it = 0; it < 200 && b - a > 4e-16 * scale; ++it) {
            const double m = 0.5 * (a + b);
            if (sturm_count(d, e, m, tiny) <= idx) a = m; else b = m;
        }
        inverse_iteration(d, e, 0.5 * (a + b), scale * 1e-18 + tiny, y);
        std::copy(y.begin(), y.end(), v.begin() + (size_t)k * N);
    }
}

// Not-a-knot cubic spline through (u_j = u0 + j D, y_j), j < N (N >= 4), evaluated at x (sorted or not).
void spline_not_a_knot(const double* yv, int N, double u0, double D, const std::vector<double>& x,
                       double* out) {
    // second derivatives M: M_{j-1} + 4 M_j + M_{j+1} = r_j (interior); not-a-knot at both ends gives
    // M_0 - 2 M_1 + M_2 = 0, which with the first interior row fixes M_1 = r_1 / 6 (uniform spacing),
    // and likewise M_{N-2} = r_{N-2} / 6.
    std::vector<double> M(N, 0.0), r(N, 0.0);
    const double s = 6.0 / (D * D);
    for (int j = 1; j + 1 < N; ++j) r[j] = s * (yv[j + 1] - 2.0 * yv[j] + yv[j - 1]);
    M[1] = r[1] / 6.0;
    M[N - 2] = r[N - 2] / 6.0;
    const int n = N - 4;  // unknowns M_2 .. M_{N-3}
    if (n > 0) {
        // tridiagonal (1, 4, 1) with the known M_1, M_{N-2} moved to the right-hand side (Thomas;
        // the matrix is strictly diagonally dominant)
        std::vector<double> c(n), g(n);
        for (int i = 0; i < n; ++i) g[i] = r[i + 2];
        g[0] -= M[1];
        g[n - 1] -= M[N - 2];
        c[0] = 1.0 / 4.0;
        g[0] /= 4.0;
        for (int i = 1; i < n; ++i) {
            const double den = 4.0 - c[i - 1];
            c[i] = 1.0 / den;
            g[i] = (g[i] - g[i - 1]) / den;
        }
        for (int i = n - 2; i >= 0; --i) g[i] -= c[i] * g[i + 1];
        for (int i = 0; i < n; ++i) M[i + 2] = g[i];
    }
    M[0] = 2.0 * M[1] - M[2];
    M[N - 1] = 2.0 * M[N - 2] - M[N - 3];
    for (size_t q = 0; q < x.size(); ++q) {
        int j = (int)std::floor((x[q] - u0) / D);
        j = std::min(std::max(j, 0), N - 2);
        const double a = u0 + (double)(j + 1) * D - x[q];  // distance to the right node
        const double b = x[q] - (u0 + (double)j * D);      // distance to the left node
        out[q] = (M[j] * a * a * a + M[j + 1] * b * b * b) / (6.0 * D) + (yv[j] / D - M[j] * D / 6.0) * a +
                 (yv[j + 1] / D - M[j + 1] * D / 6.0) * b;
    }
}

// partial[blk][k] = sum_{n in block, m < N} w_k[n] w_k[m] R(n, m) for R(B) (k < K) and R(A0) (K + k)
__global__ void quad_forms_kernel(int N, int K, const double* __restrict__ t, const double* __restrict__ w,
                                  double fmax, double fw, double* __restrict__ partial) {
    __shared__ double red[2 * kMaxK][8];
    double accB[kMaxK], accA[kMaxK];
    for (int k = 0; k < K; ++k) accB[k] = accA[k] = 0.0;
    const int n0 = blockIdx.x * kQuadRows, n1 = min(N, n0 + kQuadRows);
    for (int n = n0; n < n1; ++n) {
        const double tn = t[n];
        for (int m = threadIdx.x; m < N; m += blockDim.x) {
            double rb, ra;
            if (m == n) {
                rb = 2.0 * fmax;
                ra = 2.0 * fw;
            } else {
                const double dd = tn - t[m];
                rb = sinpi(2.0 * fmax * dd) / (kPiD * dd);
                ra = sinpi(2.0 * fw * dd) / (kPiD * dd);
            }
            for (int k = 0; k < K; ++k) {
                const double ww = w[(int64_t)k * N + n] * w[(int64_t)k * N + m];
                accB[k] += ww * rb;
                accA[k] += ww * ra;
            }
        }
    }
    // block reduction in a fixed order: warp shuffles, then the 8 warps in order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < K; ++k) {
        double b = accB[k], a = accA[k];
        for (int o = 16; o > 0; o >>= 1) {
            b += __shfl_down_sync(0xffffffffu, b, o);
            a += __shfl_down_sync(0xffffffffu, a, o);
        }
        if (lane == 0) {
            red[k][warp] = b;
            red[kMaxK + k][warp] = a;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * K) {
        const int k = threadIdx.x < K ? threadIdx.x : kMaxK + threadIdx.x - K;
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[k][q];
        partial[(int64_t)blockIdx.x * 2 * K + threadIdx.x] = s;
    }
}

}  // namespace

// ts: sorted sampling times [N]; fmax = fs / 2.  Outputs w_sorted [K][N] (order of ts) and lam [K].
m2_status spline_tapers(const std::vector<double>& ts, double fmax, double fw, int K,
                        std::vector<double>& w_sorted, std::vector<double>& lam, double& seconds) {
    const auto t0 = std::chrono::steady_clock::now();
    const int N = (int)ts.size();
    if (N < 4) {
        set_error("interpolated DPSS tapers need N >= 4 samples");
        return M2_ERR_ARG;
    }
    if (!(ts[N - 1] > ts[0])) {
        set_error("interpolated DPSS tapers need distinct first and last sampling times");
        return M2_ERR_ARG;
    }
    const double D = (ts[N - 1] - ts[0]) / (double)(N - 1);
    std::vector<double> v;
    dpss_tridiagonal(N, fw * D, K, v);  // (a)
    w_sorted.assign((size_t)K * N, 0.0);
    for (int k = 0; k < K; ++k) spline_not_a_knot(&v[(size_t)k * N], N, ts[0], D, ts, &w_sorted[(size_t)k * N]);  // (b)

    // (c) quadratic forms on the GPU
    const int nblk = (N + kQuadRows - 1) / kQuadRows;
    double *dt = nullptr, *dw = nullptr, *dp = nullptr;
    m2_status st = M2_OK;
    auto fail = [&](cudaError_t e, const char* what) {
        set_error("%s failed: %s", what, cudaGetErrorString(e));
        st = e == cudaErrorMemoryAllocation ? M2_ERR_NOMEM : M2_ERR_CUDA;
    };
    cudaError_t e = cudaMalloc(&dt, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMalloc(&dw, sizeof(double) * (size_t)K * N);
    if (e == cudaSuccess) e = cudaMalloc(&dp, sizeof(double) * (size_t)nblk * 2 * K);
    if (e != cudaSuccess) fail(e, "cudaMalloc (taper quadratic forms)");
    std::vector<double> part((size_t)nblk * 2 * K);
    if (st == M2_OK) {
        e = cudaMemcpy(dt, ts.data(), sizeof(double) * N, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(dw, w_sorted.data(), sizeof(double) * (size_t)K * N, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            quad_forms_kernel<<<nblk, 256>>>(N, K, dt, dw, fmax, fw, dp);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpy(part.data(), dp, sizeof(double) * part.size(), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) fail(e, "taper quadratic forms");
    }
    cudaFree(dt);
    cudaFree(dw);
    cudaFree(dp);
    if (st != M2_OK) return st;
    lam.assign(K, 0.0);
    for (int k = 0; k < K; ++k) {
        double qb = 0.0, qa = 0.0;
        for (int b = 0; b < nblk; ++b) {
            qb += part[(size_t)b * 2 * K + k];
            qa += part[(size_t)b * 2 * K + K + k];
        }
        if (!(qb > 0)) {
            set_error("interpolated taper %d has w^T R(B) w = %g", k, qb);
            return M2_ERR_GEP;
        }
        const double sc = std::sqrt(2.0 * fw / qb);
        for (int n = 0; n < N; ++n) w_sorted[(size_t)k * N + n] *= sc;
        lam[k] = qa / qb;
    }
    seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return M2_OK;
}

}  // namespace m2
