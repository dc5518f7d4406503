// Plan construction (Table 1 steps 1-3) and the plan-level C ABI.
//
//   * sort the sampling times, check them, detect integer grids (R(B) = I);
//   * nominal-band GEP R(A0) w = lambda R(B) w (Sec. 3.2, Eq. gep_at_A0) in
//     FP64 with cuSOLVER on matrices built by a kernel from Eq. (gpss_matrix_b)
//     and Eq. (gpss_matrix_a) with f_c0 = 0; keep the K largest eigenpairs and
//     scale to w^T R(B) w = 2 f_w (Sec. 2.2, Eq. bg_norm_requirement);
//   * NuFFT geometry: fine-grid length, support rows, split coordinates
//     (int32 cell + small offset, formed from FP64 two-products), spreading
//     tiles, twiddle tables, and the per-band deconvolution / re-phasing
//     factors (FP64 Gauss-Legendre quadrature of the kernel transform);
//   * the leakage estimate of App. B (Eq. lambda_hat_ki).
#include <cusolverDn.h>

#include <algorithm>
#include <mutex>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "packed_stages.cuh"

namespace m2 {

namespace {
thread_local std::string g_last_error;
}

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}
void clear_error() { g_last_error.clear(); }

namespace {
std::mutex g_init_mu;
bool g_init_done[64] = {};
}  // namespace

// Called with `device` current, before any exec on it.
m2_status init_device_kernels(int device) {
    if (device < 0 || device >= 64) {
        set_error("device ordinal %d out of range", device);
        return M2_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_init_mu);
    if (g_init_done[device]) return M2_OK;
    int optin = 0;
    M2_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    M2_TRY(init_exec_kernels(optin));
    M2_TRY(init_fast_kernels(optin));
    M2_TRY(init_pipe_kernels(optin));
    M2_TRY(init_hbatch_kernels(optin));
    g_init_done[device] = true;
    return M2_OK;
}

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

// exact products and sums (error-free transformations)
inline void two_prod(double a, double b, double& p, double& e) {
    p = a * b;
    e = std::fma(a, b, -p);
}
inline void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// fractional cycles of (ah + al) * t, in [-0.5, 0.5]
inline double frac_cycles(double ah, double al, double t) {
    double p, e;
    two_prod(ah, t, p, e);
    double r = (p - std::nearbyint(p)) + e + al * t;
    return r - std::nearbyint(r);
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& wt) {
    x.resize(n);
    wt.resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double dp = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = pk;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        wt[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// ---------------------------------------------------------------------------
// plan kernels (FP64)
// ---------------------------------------------------------------------------
// Column-major N x N: RB[i + j N] = sin(2 pi fmax d)/(pi d), RA likewise with f_w;
// d = t_i - t_j; diagonals 2 fmax and 2 f_w (Eqs. gpss_matrix_b, gpss_matrix_a, f_c0 = 0).
__global__ void gpss_matrices_kernel(const double* __restrict__ t, int N, double fmax, double fw,
                                     double* __restrict__ RA, double* __restrict__ RB) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= N) return;
    const size_t o = (size_t)i + (size_t)j * N;
    if (i == j) {
        RB[o] = 2.0 * fmax;
        RA[o] = 2.0 * fw;
        return;
    }
    const double d = t[i] - t[j];
    const double pd = kPi * d;
    RB[o] = sinpi(2.0 * fmax * d) / pd;
    RA[o] = sinpi(2.0 * fw * d) / pd;
}

// s[i] = exp(-i 2 pi m df t_ref) / phihat(m), m = i - i_c, with
// phihat(m) = 2 sum_q pw[q] cos(2 pi m z_q / nf)  (pw = GL weight * phi(z_q) on [0, w/2]).
template <typename C>
__global__ void deconv_kernel(int64_t I, int64_t i_c, double inv_nf, const double* __restrict__ zq,
                              const double* __restrict__ pw, int Q, double ah, double al,
                              C* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I) return;
    const double m = (double)(i - i_c);
    double acc = 0.0;
    for (int q = 0; q < Q; ++q) acc += pw[q] * cospi(2.0 * m * zq[q] * inv_nf);
    const double ph = 2.0 * acc;
    // cycles = m * (ah + al), reduced exactly
    const double p = m * ah;
    const double e = fma(m, ah, -p);
    double cyc = (p - rint(p)) + e + m * al;
    cyc -= rint(cyc);
    double s, c;
    sincospi(2.0 * cyc, &s, &c);
    C r;
    r.x = (decltype(r.x))(c / ph);
    r.y = (decltype(r.x))(-s / ph);
    out[i] = r;
}

// Integer grids: R(B) = I, so D_k^i = ||w_k||^2 for every band and
// L_k^i = lambda_k |1 - 2 f_w / ||w_k||^2| (App. B).
__global__ void leakage_const_kernel(int K, int64_t I, const double* __restrict__ Lk, double* __restrict__ L,
                                     double* __restrict__ Eh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I) return;
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        L[(int64_t)k * I + i] = Lk[k];
        s += Lk[k];
    }
    Eh[i] = s / K;
}

// Sub-band plans (complex tapers w = a + i b, band B^q = {f_min <= |f| <= f_max}, shifts
// df_i = f_ci - f_c0), small problems: the same estimate with R(B^q) (App. B with Eq.
// gpss_matrix_b_q):  D_k^i = sum_{n,m} Re[conj(w_n) w_m e^{-i 2 pi df_i (t_n - t_m)}] R(B^q|n,m)
//   = sum_n |w_n|^2 R_nn + 2 sum_{n<m} [(a_n a_m + b_n b_m) cos(th) + (a_n b_m - b_n a_m) sin(th)] R_nm,
// th = 2 pi df_i (t_n - t_m), R_nm = 2 cos(pi (f_max + f_min) d) sin(pi (f_max - f_min) d) / (pi d),
// R_nn = 2 (f_max - f_min).  One CTA per band, fixed-order reduction, as leakage_direct_kernel.
constexpr int kLeakThreadsC = 256;
__global__ void __launch_bounds__(kLeakThreadsC) leakage_direct_cplx_kernel(
    int N, int K, int64_t I, const double* __restrict__ tc, const double* __restrict__ wr /*[K][N] sorted*/,
    const double* __restrict__ wi, double f_min, double f_max, double f_lo, double df,
    const double* __restrict__ lam, double fw, double* __restrict__ L, double* __restrict__ Eh) {
    __shared__ double s_red[kLeakThreadsC];
    __shared__ double s_D[kMaxK];
    const int64_t i = blockIdx.x;
    const double f = f_lo + (double)i * df;
    double D[kMaxK];
    for (int k = 0; k < K; ++k) D[k] = 0.0;
    const double rnn = 2.0 * (f_max - f_min);
    for (int n = threadIdx.x; n < N; n += kLeakThreadsC) {
        const double tn = tc[n];
        for (int k = 0; k < K; ++k) {
            const double a = wr[(int64_t)k * N + n], b = wi[(int64_t)k * N + n];
            D[k] += (a * a + b * b) * rnn;
        }
        for (int m = n + 1; m < N; ++m) {
            const double d = tn - tc[m];
            const double r = 2.0 * cospi((f_max + f_min) * d) * sinpi((f_max - f_min) * d) / (kPi * d) * 2.0;
            double sn, cs;
            sincospi(2.0 * f * d, &sn, &cs);
            for (int k = 0; k < K; ++k) {
                const double an = wr[(int64_t)k * N + n], bn = wi[(int64_t)k * N + n];
                const double am = wr[(int64_t)k * N + m], bm = wi[(int64_t)k * N + m];
                D[k] += ((an * am + bn * bm) * cs + (an * bm - bn * am) * sn) * r;
            }
        }
    }
    for (int k = 0; k < K; ++k) {
        s_red[threadIdx.x] = D[k];
        __syncthreads();
        for (int h = kLeakThreadsC / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) s_red[threadIdx.x] += s_red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) s_D[k] = s_red[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) {
            const double lh = lam[k] * 2.0 * fw / s_D[k];
            const double l = fabs(lam[k] - lh);
            L[(int64_t)k * I + i] = l;
            s += l;
        }
        Eh[i] = s / K;
    }
}

// General sampling, small problems: D_k^i = sum_{n,m} w_n w_m R(B|n,m) cos(2 pi f_i (t_n - t_m))
// evaluated directly (App. B, Eq. lambda_hat_ki).  One CTA per band: the threads split the rows n
// (n = tid, tid + blockDim, ...; row n adds the diagonal term and twice the pairs m > n), then a
// fixed-order tree reduction over the CTA gives D_k, so the result is the same on every run.
constexpr int kLeakThreads = 256;
__global__ void __launch_bounds__(kLeakThreads) leakage_direct_kernel(
    int N, int K, int64_t I, const double* __restrict__ tc, const double* __restrict__ w /*[K][N] sorted*/,
    double fmax, double f_lo, double df, const double* __restrict__ lam, double fw, double* __restrict__ L,
    double* __restrict__ Eh) {
    __shared__ double s_red[kLeakThreads];
    __shared__ double s_D[kMaxK];
    const int64_t i = blockIdx.x;
    const double f = f_lo + (double)i * df;
    double D[kMaxK];
    for (int k = 0; k < K; ++k) D[k] = 0.0;
    for (int n = threadIdx.x; n < N; n += kLeakThreads) {
        const double tn = tc[n];
        for (int k = 0; k < K; ++k) D[k] += w[(int64_t)k * N + n] * w[(int64_t)k * N + n] * 2.0 * fmax;
        for (int m = n + 1; m < N; ++m) {
            const double d = tn - tc[m];
            const double r = sinpi(2.0 * fmax * d) / (kPi * d) * 2.0 * cospi(2.0 * f * d);
            for (int k = 0; k < K; ++k) D[k] += w[(int64_t)k * N + n] * w[(int64_t)k * N + m] * r;
        }
    }
    for (int k = 0; k < K; ++k) {
        s_red[threadIdx.x] = D[k];
        __syncthreads();
        for (int h = kLeakThreads / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) s_red[threadIdx.x] += s_red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) s_D[k] = s_red[0];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) {
            const double lh = lam[k] * 2.0 * fw / s_D[k];
            const double l = fabs(lam[k] - lh);
            L[(int64_t)k * I + i] = l;
            s += l;
        }
        Eh[i] = s / K;
    }
}

// Windowed leakage (general sampling at scale).  R(B|n,m) is the integral of
// exp(i 2 pi nu (t_n - t_m)) over the signal band (Eq. gpss_matrix_b), so
//   D_k(f) = integral over [f - f_max, f + f_max] of |W_k(phi)|^2 dphi,
//   W_k(phi) = sum_n w_k(t_n) exp(-i 2 pi phi t_n).
// |W_k|^2 is band-limited (its "time" support is |tau| <= T, the sampling
// span), so sampled on a grid with spacing delta < 1/(2T) it is reproduced
// exactly by a smooth band-limited interpolator; integrating that interpolant
// over each window gives weight delta for interior samples and tabulated edge
// weights within M samples of the two ends.
// G[k][j] = |W_k(phi_j)|^2 and S[k][j] = sum_{q < j} G[k][q] (one CTA per taper).
__global__ void leak_prefix_kernel(int64_t Jn, const double2* __restrict__ Wv, double* __restrict__ G,
                                   double* __restrict__ S) {
    __shared__ double s_part[1024];
    const int k = blockIdx.x;
    const double2* Wk = Wv + (int64_t)k * Jn;
    double* Gk = G + (int64_t)k * Jn;
    double* Sk = S + (int64_t)k * (Jn + 1);
    const int64_t per = (Jn + blockDim.x - 1) / blockDim.x;
    const int64_t j0 = (int64_t)threadIdx.x * per, j1 = min(Jn, j0 + per);
    double acc = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        const double2 v = Wk[j];
        const double g = v.x * v.x + v.y * v.y;
        Gk[j] = g;
        acc += g;
    }
    s_part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {  // fixed-order exclusive scan of the segment sums
        double run = 0.0;
        for (int q = 0; q < (int)blockDim.x; ++q) {
            const double v = s_part[q];
            s_part[q] = run;
            run += v;
        }
        Sk[Jn] = run;
    }
    __syncthreads();
    double run = s_part[threadIdx.x];
    for (int64_t j = j0; j < j1; ++j) {
        Sk[j] = run;
        run += Gk[j];
    }
}

// D_k(f_i) from the prefix sums and the edge weights; then L-hat / E-hat.
__global__ void leak_window_kernel(int K, int64_t I, int64_t Jn, int r, int M, int Wi, double delta,
                                   const double* __restrict__ G, const double* __restrict__ S,
                                   const double* __restrict__ left /*[2M-1], p = -M+1..M-1*/,
                                   const double* __restrict__ right /*[2M], p = Wi-M+1..Wi+M*/,
                                   const double* __restrict__ lam, double fw, double* __restrict__ L,
                                   double* __restrict__ Eh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I) return;
    const int64_t base = M + i * r;
    double sum = 0.0;
    for (int k = 0; k < K; ++k) {
        const double* Gk = G + (int64_t)k * Jn;
        const double* Sk = S + (int64_t)k * (Jn + 1);
        double D = delta * (Sk[base + Wi - M + 1] - Sk[base + M]);
        for (int q = 0; q < 2 * M - 1; ++q) D += left[q] * Gk[base - M + 1 + q];
        for (int q = 0; q < 2 * M; ++q) D += right[q] * Gk[base + Wi - M + 1 + q];
        const double lh = lam[k] * 2.0 * fw / D;
        const double l = fabs(lam[k] - lh);
        L[(int64_t)k * I + i] = l;
        sum += l;
    }
    Eh[i] = sum / K;
}

// fill a device array with ones (the unit signal whose eigencoefficients are the taper transforms)
__global__ void ones_kernel(double* v, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = 1.0;
}

// ---------------------------------------------------------------------------
// device allocation helpers
// ---------------------------------------------------------------------------
struct PlanBuilder {
    m2nufft_plan_s* p;
    size_t budget;
    template <typename T>
    m2_status alloc(T** out, size_t count) {
        size_t bytes = std::max<size_t>(count * sizeof(T), 16);
        if (budget && p->device_bytes + bytes > budget) {
            set_error("plan needs more than mem_budget = %zu bytes of device memory", budget);
            return M2_ERR_BUDGET;
        }
        void* d = nullptr;
        cudaError_t e = cudaMalloc(&d, bytes);
        if (e != cudaSuccess) {
            set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
            return M2_ERR_NOMEM;
        }
        p->allocations.push_back(d);
        p->device_bytes += bytes;
        *out = reinterpret_cast<T*>(d);
        return M2_OK;
    }
    template <typename T>
    m2_status upload(T** out, const std::vector<T>& h) {
        M2_TRY(alloc(out, h.size()));
        M2_CUDA_TRY(cudaMemcpy(*out, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
        return M2_OK;
    }
};

void free_plan(m2nufft_plan_s* p) {
    if (!p) return;
    purge_batch_graphs(p);
    {
        DeviceGuard guard(p->device);
        cudaDeviceSynchronize();
        for (auto& kv : p->pipe_cache) pipe_free(kv.second);
        for (int L = 0; L < kLanes; ++L) {
            if (p->lane_st[L]) cudaStreamDestroy(p->lane_st[L]);
            if (p->lane_ev[L]) cudaEventDestroy(p->lane_ev[L]);
        }
        if (p->fork_ev) cudaEventDestroy(p->fork_ev);
        if (p->d_gall) cudaFree(p->d_gall);
        if (p->gall_ev) cudaEventDestroy(p->gall_ev);
        if (p->pipe_status) cudaFreeHost(p->pipe_status);
        if (p->stage_status) cudaFreeHost(p->stage_status);
        if (p->d_pipe_prof) cudaFree(p->d_pipe_prof);
        for (void* d : p->allocations) cudaFree(d);
        for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
        for (auto& kk : p->ev_rec)
            for (auto& v : kk)
                for (cudaEvent_t e : v) cudaEventDestroy(e);
    }
    delete p;
}

// ---------------------------------------------------------------------------
// GEP on the GPU (cuSOLVER, FP64)
// ---------------------------------------------------------------------------
m2_status solve_gep(const std::vector<double>& ts, double fmax, double fw, int K, size_t budget,
                    std::vector<double>& w_sorted, std::vector<double>& lam, double& seconds) {
    const int N = (int)ts.size();
    auto t0 = std::chrono::steady_clock::now();
    const size_t mat = (size_t)N * N;
    double *dA = nullptr, *dB = nullptr, *dt = nullptr, *dW = nullptr, *work = nullptr;
    int* dinfo = nullptr;
    cusolverDnHandle_t h = nullptr;
    m2_status st = M2_OK;
    int lwork = 0, meig = 0, info = 0;
    cusolverStatus_t cs;

    auto fail = [&](m2_status s) {
        st = s;
    };
    do {
        if (budget && 2 * mat * sizeof(double) > budget) {
            set_error("GEP needs %zu bytes for R(A0) and R(B), above mem_budget", 2 * mat * sizeof(double));
            fail(M2_ERR_BUDGET);
            break;
        }
        cudaError_t e;
        if ((e = cudaMalloc(&dA, mat * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&dB, mat * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&dt, N * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&dW, N * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&dinfo, sizeof(int))) != cudaSuccess) {
            set_error("GEP allocation failed: %s", cudaGetErrorString(e));
            fail(M2_ERR_NOMEM);
            break;
        }
        if ((e = cudaMemcpy(dt, ts.data(), N * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) {
            set_error("GEP copy failed: %s", cudaGetErrorString(e));
            fail(M2_ERR_CUDA);
            break;
        }
        dim3 grid((N + 255) / 256, N);
        gpss_matrices_kernel<<<grid, 256>>>(dt, N, fmax, fw, dA, dB);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            set_error("GPSS matrix kernel failed: %s", cudaGetErrorString(e));
            fail(M2_ERR_CUDA);
            break;
        }
        if ((cs = cusolverDnCreate(&h)) != CUSOLVER_STATUS_SUCCESS) {
            set_error("cusolverDnCreate failed (%d)", (int)cs);
            fail(M2_ERR_CUDA);
            break;
        }
        cs = cusolverDnDsygvdx_bufferSize(h, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                                          CUBLAS_FILL_MODE_LOWER, N, dA, N, dB, N, 0.0, 0.0, N - K + 1, N,
                                          &meig, dW, &lwork);
        if (cs != CUSOLVER_STATUS_SUCCESS) {
            set_error("cusolverDnDsygvdx_bufferSize failed (%d)", (int)cs);
            fail(M2_ERR_GEP);
            break;
        }
        if (budget && (2 * mat + (size_t)lwork) * sizeof(double) > budget) {
            set_error("GEP workspace exceeds mem_budget");
            fail(M2_ERR_BUDGET);
            break;
        }
        if ((e = cudaMalloc(&work, sizeof(double) * std::max(lwork, 1))) != cudaSuccess) {
            set_error("GEP workspace allocation failed: %s", cudaGetErrorString(e));
            fail(M2_ERR_NOMEM);
            break;
        }
        cs = cusolverDnDsygvdx(h, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                               CUBLAS_FILL_MODE_LOWER, N, dA, N, dB, N, 0.0, 0.0, N - K + 1, N, &meig, dW,
                               work, lwork, dinfo);
        if (cs != CUSOLVER_STATUS_SUCCESS) {
            set_error("cusolverDnDsygvdx failed (%d)", (int)cs);
            fail(M2_ERR_GEP);
            break;
        }
        if ((e = cudaMemcpy(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess) {
            set_error("GEP info copy failed: %s", cudaGetErrorString(e));
            fail(M2_ERR_CUDA);
            break;
        }
        if (info != 0) {
            if (info > N)
                set_error("R(B) is not positive definite in FP64 (cuSOLVER info %d): "
                          "sampling times too close or repeated",
                          info);
            else
                set_error("GEP did not converge (cuSOLVER info %d)", info);
            fail(M2_ERR_GEP);
            break;
        }
        if (meig != K) {
            set_error("GEP returned %d eigenpairs, expected %d", meig, K);
            fail(M2_ERR_GEP);
            break;
        }
        std::vector<double> W(K), V((size_t)K * N);
        if ((e = cudaMemcpy(W.data(), dW, K * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(V.data(), dA, (size_t)K * N * sizeof(double), cudaMemcpyDeviceToHost)) !=
                cudaSuccess) {
            set_error("GEP result copy failed: %s", cudaGetErrorString(e));
            fail(M2_ERR_CUDA);
            break;
        }
        // ascending -> descending; eigenvectors satisfy v^T R(B) v = 1, so scale by sqrt(2 f_w)
        const double sc = std::sqrt(2.0 * fw);
        lam.assign(K, 0.0);
        w_sorted.assign((size_t)K * N, 0.0);
        for (int k = 0; k < K; ++k) {
            const int src = K - 1 - k;
            lam[k] = W[src];
            for (int n = 0; n < N; ++n) w_sorted[(size_t)k * N + n] = V[(size_t)src * N + n] * sc;
        }
    } while (0);
    if (h) cusolverDnDestroy(h);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dt);
    cudaFree(dW);
    cudaFree(work);
    cudaFree(dinfo);
    cudaDeviceSynchronize();
    seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

int64_t next_pow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}
int ilog2(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

// Kcum(x) = integral_{-inf}^{x} kappa(u) du for the band-limited interpolator with transform
// kappa_hat(tau) = delta psi(tau): psi = 1 for |tau| <= Tb, an erfc roll-off to 0 at tau_c = 1/delta - Tb.
double kcum(double x, double delta, double Tb, const std::vector<double>& gx, const std::vector<double>& gw) {
    const double tau_c = 1.0 / delta - Tb;
    const double sig = (tau_c - Tb) / 16.0, mid = 0.5 * (Tb + tau_c);
    double acc = 0.0;
    for (size_t q = 0; q < gx.size(); ++q) {
        const double tau = 0.5 * (gx[q] + 1.0) * tau_c;
        const double psi = tau <= Tb ? 1.0 : 0.5 * std::erfc((tau - mid) / (std::sqrt(2.0) * sig));
        acc += 0.5 * tau_c * gw[q] * psi * std::sin(2.0 * kPi * x * tau) / (kPi * tau);
    }
    return delta * (0.5 + acc);
}

// L-hat / E-hat for general sampling at scale (see leak_window_kernel).
m2_status windowed_leakage(m2nufft_plan_s* p, const std::vector<double>& ts) {
    const Geometry& g = p->g;
    const int K = g.K;
    const int64_t N = g.N, I = g.I;
    const double fmax = 0.5 * p->fs;
    const double T = std::max(ts.back() - ts.front(), 1e-300);
    const int r = (int)std::max<double>(1.0, std::ceil(3.0 * T * g.df));  // delta <= 1/(3T)
    const double delta = g.df / r;
    const int M = 48;
    const double Wd = 2.0 * fmax / delta;
    const int Wi = (int)std::floor(Wd);
    if (Wi < 2 * M + 2) {
        set_error("windowed leakage needs fs/delta >= %d", 2 * M + 2);
        return M2_ERR_ARG;
    }
    const int64_t Jn = (I - 1) * r + Wi + 2 * M + 2;
    const double phi0 = g.f_lo - fmax - M * delta;

    // edge weights
    std::vector<double> gx, gw;
    gauss_legendre(2000, gx, gw);
    std::vector<double> left(2 * M - 1), right(2 * M);
    for (int q = 0; q < 2 * M - 1; ++q) {
        const int pp = -M + 1 + q;
        left[q] = delta - kcum(-pp * delta, delta, T, gx, gw);
    }
    for (int q = 0; q < 2 * M; ++q) {
        const int pp = Wi - M + 1 + q;
        right[q] = kcum((Wd - pp) * delta, delta, T, gx, gw);
    }

    // W_k on the extended grid with the library's FP64 NuFFT (a temporary plan with the same tapers)
    m2_fgrid fg{phi0, delta, Jn};
    m2_opts o{};
    o.precision = 64;
    o.tol = 1e-13;
    o.device = p->device;
    o.max_batch = 1;
    o.path = 1;
    m2nufft_plan_t tp = nullptr;
    m2_status st = m2nufft_plan_with_tapers(p->t.data(), N, p->fs, p->f_w, K, &fg, p->w.data(), nullptr, &o, &tp);
    if (st != M2_OK) return st;
    double *d_x = nullptr, *d_G = nullptr, *d_S = nullptr, *d_l = nullptr, *d_r = nullptr, *d_lam = nullptr;
    double2* d_W = nullptr;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
        cudaFree(d_x);
        cudaFree(d_G);
        cudaFree(d_S);
        cudaFree(d_l);
        cudaFree(d_r);
        cudaFree(d_lam);
        cudaFree(d_W);
        m2nufft_destroy(tp);
    };
    if ((e = cudaMalloc(&d_x, sizeof(double) * N)) != cudaSuccess ||
        (e = cudaMalloc(&d_W, sizeof(double2) * K * Jn)) != cudaSuccess ||
        (e = cudaMalloc(&d_G, sizeof(double) * K * Jn)) != cudaSuccess ||
        (e = cudaMalloc(&d_S, sizeof(double) * K * (Jn + 1))) != cudaSuccess ||
        (e = cudaMalloc(&d_l, sizeof(double) * left.size())) != cudaSuccess ||
        (e = cudaMalloc(&d_r, sizeof(double) * right.size())) != cudaSuccess ||
        (e = cudaMalloc(&d_lam, sizeof(double) * K)) != cudaSuccess) {
        cleanup();
        set_error("windowed leakage allocation failed: %s", cudaGetErrorString(e));
        return M2_ERR_NOMEM;
    }
    cudaMemcpy(d_l, left.data(), sizeof(double) * left.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(d_r, right.data(), sizeof(double) * right.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(d_lam, p->lambda.data(), sizeof(double) * K, cudaMemcpyHostToDevice);
    ones_kernel<<<(unsigned)((N + 255) / 256), 256>>>(d_x, N);
    st = m2nufft_exec(tp, d_x, 1, d_W, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (st != M2_OK) {
        cleanup();
        return st;
    }
    leak_prefix_kernel<<<K, 1024>>>(Jn, d_W, d_G, d_S);
    leak_window_kernel<<<(unsigned)((I + 127) / 128), 128>>>(K, I, Jn, r, M, Wi, delta, d_G, d_S, d_l, d_r, d_lam,
                                                             p->f_w, p->d_Lhat, p->d_Ehat);
    e = cudaDeviceSynchronize();
    cleanup();
    if (e != cudaSuccess) {
        set_error("windowed leakage kernels failed: %s", cudaGetErrorString(e));
        return M2_ERR_CUDA;
    }
    return M2_OK;
}

template <typename R>
m2_status upload_typed(PlanBuilder& pb, void** out, const std::vector<double>& h) {
    std::vector<R> v(h.begin(), h.end());
    R* d = nullptr;
    M2_TRY(pb.upload(&d, v));
    *out = d;
    return M2_OK;
}

// complex table stored as interleaved (re, im) doubles -> precision-typed device copy
m2_status upload_complex(PlanBuilder& pb, int precision, void** out, const std::vector<double>& h) {
    return precision == 32 ? upload_typed<float>(pb, out, h) : upload_typed<double>(pb, out, h);
}

std::vector<double> unit_roots(int64_t count, int64_t n, int64_t step) {
    // exp(-i 2 pi (q * step) / n), q < count
    std::vector<double> v(2 * count);
    for (int64_t q = 0; q < count; ++q) {
        const int64_t a = (q * step) % n;
        const double x = 2.0 * (double)a / (double)n;  // angle / pi, exact
        v[2 * q] = std::cos(kPi * x);
        v[2 * q + 1] = -std::sin(kPi * x);
    }
    return v;
}

#define M2_TRY_OR(expr)                   \
    do {                                  \
        m2_status s_ = (expr);            \
        if (s_ != M2_OK) return bail(s_); \
    } while (0)
#define M2_CUDA_TRY_OR(expr)                                                                 \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return bail(e_ == cudaErrorMemoryAllocation ? M2_ERR_NOMEM : M2_ERR_CUDA);        \
        }                                                                                    \
    } while (0)

m2_status build_plan(const double* t, int64_t N, double fs, double f_w, int K, const m2_fgrid* fc,
                     const double* w_given, const double* lam_given, const m2_opts* opts_in,
                     m2nufft_plan_t* out, const m2_subband* sb = nullptr, const double* wc_given = nullptr) {
    if (!out) {
        set_error("out is NULL");
        return M2_ERR_ARG;
    }
    *out = nullptr;
    m2_opts opts{};
    opts.precision = 32;
    if (opts_in) opts = *opts_in;
    if (opts.precision != 32 && opts.precision != 64) {
        set_error("precision must be 32 or 64");
        return M2_ERR_ARG;
    }
    if (!t || N < 1 || N > (int64_t(1) << 30)) {
        set_error("need t != NULL and 1 <= N <= 2^30");
        return M2_ERR_ARG;
    }
    if (!(fs > 0) || !std::isfinite(fs)) {
        set_error("fs must be positive and finite");
        return M2_ERR_ARG;
    }
    const double fmax = 0.5 * fs;
    if (!(f_w > 0) || !(f_w < fmax)) {
        set_error("need 0 < f_w < fs/2");
        return M2_ERR_ARG;
    }
    if (K < 1 || K > kMaxK || K > N) {
        set_error("need 1 <= K <= min(N, %d)", kMaxK);
        return M2_ERR_ARG;
    }
    if (!fc || fc->I < 1 || fc->I > (int64_t(1) << 23) || !(fc->df > 0) || !std::isfinite(fc->df) ||
        !std::isfinite(fc->f_lo)) {
        set_error("band grid needs 1 <= I <= 2^23, df > 0 and finite f_lo");
        return M2_ERR_ARG;
    }
    for (int64_t n = 0; n < N; ++n) {
        if (!std::isfinite(t[n])) {
            set_error("sampling time %lld is not finite", (long long)n);
            return M2_ERR_ARG;
        }
    }
    // sub-band B^q = {f_min <= |f| <= f_max} and nominal centre f_c0 (Sec. 2.3, Sec. 3 multiband partition)
    const bool cplx = sb != nullptr;
    const double f_c0 = cplx ? sb->f_c0 : 0.0;
    if (cplx) {
        const double a = std::fabs(sb->f_c0);
        const bool inside = sb->f_min == 0.0 ? (a + f_w <= sb->f_max) : (sb->f_min <= a - f_w && a + f_w <= sb->f_max);
        if (!(sb->f_min >= 0) || !(sb->f_max > sb->f_min) || !(sb->f_max <= fmax) || !std::isfinite(sb->f_c0) ||
            !inside) {
            set_error("sub-band needs 0 <= f_min < f_max <= fs/2 and the nominal band |f - f_c0| <= f_w inside "
                      "f_min <= |f| <= f_max");
            return M2_ERR_ARG;
        }
    }
    if (wc_given) {
        for (int64_t q = 0; q < 2 * (int64_t)K * N; ++q)
            if (!std::isfinite(wc_given[q])) {
                set_error("taper value %lld is not finite", (long long)q);
                return M2_ERR_ARG;
            }
    }
    // band centres relative to the nominal centre: Delta f_i = f_ci - f_c0 (Eq. freq_shift_op)
    m2_fgrid fcs = *fc;
    fcs.f_lo = fc->f_lo - f_c0;
    fc = &fcs;
    if (w_given) {
        for (int64_t q = 0; q < (int64_t)K * N; ++q)
            if (!std::isfinite(w_given[q])) {
                set_error("taper value %lld is not finite", (long long)q);
                return M2_ERR_ARG;
            }
    }

    int dev = opts.device;
    if (dev < 0) M2_CUDA_TRY(cudaGetDevice(&dev));
    DeviceGuard guard(dev);
    M2_TRY(init_device_kernels(dev));

    int nsm = 0;
    M2_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    auto* p = new m2nufft_plan_s();
    p->device = dev;
    p->sm_count = nsm;
    p->precision = opts.precision;
    p->fs = fs;
    p->f_w = f_w;
    p->tol = opts.tol > 0 ? opts.tol : (opts.precision == 32 ? 1e-6 : 1e-12);
    p->t.assign(t, t + N);
    PlanBuilder pb{p, opts.mem_budget};
    auto bail = [&](m2_status s) {
        free_plan(p);
        return s;
    };

    // ---- sort ----
    std::vector<int64_t> ord(N);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return t[a] < t[b]; });
    std::vector<double> ts(N);
    for (int64_t j = 0; j < N; ++j) ts[j] = t[ord[j]];
    bool integer_grid = true;
    for (int64_t j = 0; j < N; ++j) {
        const double v = ts[j] * fs;
        if (v != std::nearbyint(v) || std::fabs(v) > 9.0e15) {
            integer_grid = false;
            break;
        }
    }
    p->integer_grid = integer_grid ? 1 : 0;

    // ---- tapers ----
    std::vector<double> w_sorted((size_t)K * N), w_sorted_im;  // imaginary parts: sub-band plans only
    if (cplx) {
        w_sorted_im.assign((size_t)K * N, 0.0);
        if (wc_given) {
            for (int k = 0; k < K; ++k)
                for (int64_t j = 0; j < N; ++j) {
                    w_sorted[(size_t)k * N + j] = wc_given[2 * ((size_t)k * N + ord[j])];
                    w_sorted_im[(size_t)k * N + j] = wc_given[2 * ((size_t)k * N + ord[j]) + 1];
                }
            if (lam_given) {
                p->lambda.assign(lam_given, lam_given + K);
                p->have_lambda = 1;
            }
        } else {
            for (int64_t j = 0; j + 1 < N; ++j)
                if (ts[j] == ts[j + 1]) {
                    set_error("repeated sampling time %.17g: R(B^q) is singular", ts[j]);
                    return bail(M2_ERR_GEP);
                }
            if (N > 46340) {
                set_error("GEP size N = %lld is above the dense solver limit (46340)", (long long)N);
                return bail(M2_ERR_ARG);
            }
            std::vector<double> lam;
            m2_status s = solve_gep_subband(ts, f_w, K, f_c0, sb->f_min, sb->f_max, opts.mem_budget, w_sorted,
                                            w_sorted_im, lam, p->gep_seconds);
            if (s != M2_OK) return bail(s);
            // phase: sum_n w_k(t_n) e^{-i 2 pi f_c0 t_n} (t_n - tbar)^(k mod 2) real and positive
            double tbar = 0;
            for (double v : ts) tbar += v;
            tbar /= (double)N;
            for (int k = 0; k < K; ++k) {
                double sr = 0, si = 0;
                for (int64_t j = 0; j < N; ++j) {
                    const double cyc = frac_cycles(-f_c0, 0.0, ts[j]);
                    const double c = std::cos(2.0 * kPi * cyc), sn = std::sin(2.0 * kPi * cyc);
                    const double fac = (k & 1) ? (ts[j] - tbar) : 1.0;
                    const double wr = w_sorted[(size_t)k * N + j], wi = w_sorted_im[(size_t)k * N + j];
                    sr += fac * (wr * c - wi * sn);
                    si += fac * (wr * sn + wi * c);
                }
                const double a = std::hypot(sr, si);
                if (a > 0) {
                    const double cr = sr / a, ci = -si / a;  // multiply by conj(S) / |S|
                    for (int64_t j = 0; j < N; ++j) {
                        const double wr = w_sorted[(size_t)k * N + j], wi = w_sorted_im[(size_t)k * N + j];
                        w_sorted[(size_t)k * N + j] = wr * cr - wi * ci;
                        w_sorted_im[(size_t)k * N + j] = wr * ci + wi * cr;
                    }
                }
            }
            p->lambda = lam;
            p->have_lambda = 1;
        }
    } else if (w_given) {
        for (int k = 0; k < K; ++k)
            for (int64_t j = 0; j < N; ++j) w_sorted[(size_t)k * N + j] = w_given[(size_t)k * N + ord[j]];
        if (lam_given) {
            p->lambda.assign(lam_given, lam_given + K);
            p->have_lambda = 1;
        }
    } else {
        for (int64_t j = 0; j + 1 < N; ++j)
            if (ts[j] == ts[j + 1]) {
                set_error("repeated sampling time %.17g: R(B) is singular", ts[j]);
                return bail(M2_ERR_GEP);
            }
        if (opts.tapers != 0 && opts.tapers != 1) {
            set_error("opts.tapers must be 0 (GEP) or 1 (interpolated DPSS)");
            return bail(M2_ERR_ARG);
        }
        std::vector<double> lam;
        if (opts.tapers == 1) {
            // Table 1 step 3 (a)-(c): DPSS on a uniform grid, cubic spline to t, R(B) normalisation
            m2_status s = spline_tapers(ts, fmax, f_w, K, w_sorted, lam, p->gep_seconds);
            if (s != M2_OK) return bail(s);
        } else {
            if (N > 46340) {
                set_error("GEP size N = %lld is above the dense solver limit (46340)", (long long)N);
                return bail(M2_ERR_ARG);
            }
            m2_status s = solve_gep(ts, fmax, f_w, K, opts.mem_budget, w_sorted, lam, p->gep_seconds);
            if (s != M2_OK) return bail(s);
        }
        // sign: sum_n w_k(t_n) (t_n - tbar)^(k mod 2) > 0
        double tbar = 0;
        for (double v : ts) tbar += v;
        tbar /= (double)N;
        for (int k = 0; k < K; ++k) {
            double sgn = 0;
            for (int64_t j = 0; j < N; ++j) sgn += w_sorted[(size_t)k * N + j] * ((k & 1) ? (ts[j] - tbar) : 1.0);
            if (sgn < 0)
                for (int64_t j = 0; j < N; ++j) w_sorted[(size_t)k * N + j] = -w_sorted[(size_t)k * N + j];
        }
        p->lambda = lam;
        p->have_lambda = 1;
    }
    p->w.assign((size_t)K * N, 0.0);
    for (int k = 0; k < K; ++k)
        for (int64_t j = 0; j < N; ++j) p->w[(size_t)k * N + ord[j]] = w_sorted[(size_t)k * N + j];
    p->complex_taper = cplx ? 1 : 0;
    p->f_c0 = f_c0;
    if (cplx) {
        p->w_im.assign((size_t)K * N, 0.0);
        for (int k = 0; k < K; ++k)
            for (int64_t j = 0; j < N; ++j) p->w_im[(size_t)k * N + ord[j]] = w_sorted_im[(size_t)k * N + j];
    }

    // ---- geometry ----
    Geometry& g = p->g;
    g.N = N;
    g.K = K;
    g.I = fc->I;
    g.f_lo = fc->f_lo;
    g.df = fc->df;
    g.i_c = g.I / 2;
    {
        double pr, pe, s, se;
        two_prod((double)g.i_c, g.df, pr, pe);
        two_sum(g.f_lo, pr, s, se);
        g.fmid_hi = s;
        g.fmid_lo = se + pe;
    }
    double tmax_abs = 0;
    for (double v : ts) tmax_abs = std::max(tmax_abs, std::fabs(v));
    // the modulation exp(-i 2 pi f_mid t) is dropped when its phase stays below a threshold over the
    // whole span: 1e-9 cycles for FP32 plans (relative effect <= 6.3e-9, far below their tolerance; a
    // grid like f_lo = -1/2, df = 1/I leaves f_mid = O(1e-16) from the rounding of df), 1e-12 for FP64
    const double real_thresh = opts.precision == 32 ? 1e-9 : 1e-12;
    g.real_taper = !cplx && (std::fabs(g.fmid_hi) + std::fabs(g.fmid_lo)) * tmax_abs < real_thresh ? 1 : 0;
    // ---- exec path, fine-grid length and spreading kernel ----
    // generic path: nf = power of two >= 2 I (sigma in [2, 4)), w = ceil(log10(1/tol)) + 1, beta = 2.30 w.
    // packed FP32 path: nf = smallest 2^a or 3 * 2^a >= 1.5 I (sigma in [1.5, 2)), w = ceil(1.25 log10(1/tol))
    // + 1; with opts.sigma in [1.25, 1.5) also nf = 5 * 2^a, and below sigma 1.5
    // w = ceil(ln(1/tol) / (pi sqrt(1 - 1/sigma))) + 1 (11 at sigma 1.25, tol 1e-6; the same rule gives
    // the 9 of the first one at 1.5); beta = 0.97 pi (1 - 1/(2 sigma)) w (exponential-of-semicircle
    // kernel, Barnett et al. 2019).
    if (opts.path < 0 || opts.path > 3) {
        set_error("opts.path must be 0, 1, 2 or 3");
        return bail(M2_ERR_ARG);
    }
    const double span_t = ts.back() - ts.front();
    bool packed_ok = false;
    int64_t nf_packed = 0;
    if (!(opts.sigma == 0.0 || (opts.sigma >= 1.25 && opts.sigma <= 8.0))) {
        set_error("opts.sigma must be 0 (automatic) or in [1.25, 8]");
        return bail(M2_ERR_ARG);
    }
    int w_packed = 0;
    if (opts.precision == 32 && g.real_taper && opts.path != 1) {
        // nf >= sigma I with sigma = 1.5 unless asked otherwise; at sigma >= 2 the kernel needs the
        // narrower width of the generic rule
        const double target = std::max((opts.sigma > 0 ? opts.sigma : 1.5) * (double)g.I, 2048.0);
        int64_t a2 = 2048, a3 = 3 * 2048, a5 = 5 * 2048;  // nf = 1024 * n1 with n1 even
        while ((double)a2 < target) a2 <<= 1;
        while ((double)a3 < target) a3 <<= 1;
        while ((double)a5 < target) a5 <<= 1;
        nf_packed = std::min(a2, a3);
        if (opts.sigma > 0 && opts.sigma < 1.5) nf_packed = std::min(nf_packed, a5);
        const double sig = (double)nf_packed / (double)g.I;
        if (sig >= 2.0)
            w_packed = std::min(16, std::max(2, (int)std::ceil(std::log10(1.0 / p->tol)) + 1));
        else if (sig >= 1.5)
            w_packed = std::min(16, std::max(2, (int)std::ceil(1.25 * std::log10(1.0 / p->tol)) + 1));
        else
            w_packed = std::min(16, std::max(2, (int)std::ceil(std::log(1.0 / p->tol) /
                                                               (kPi * std::sqrt(1.0 - 1.0 / sig))) + 1));
        const double span = span_t * (double)nf_packed * g.df;
        const bool wrap_p = span + w_packed + 2.0 >= (double)nf_packed;
        const int64_t rows_p = wrap_p ? nf_packed / 1024 : (int64_t)std::ceil((span + w_packed + 2.0) / 1024.0);
        packed_ok = nf_packed % 2048 == 0 && nf_packed <= (int64_t(3) << 20) && rows_p <= 64;
    }
    if (opts.path >= 2 && !packed_ok) {
        set_error("the packed FP32 path needs precision 32, a real modulated taper (f_lo + (I/2) df = 0), "
                  "I <= 2^21 and a support of at most 64 rows of 1024 cells");
        return bail(M2_ERR_ARG);
    }
    // packed plans run the four-kernel form (2) unless the persistent pipelined kernel (3) is asked for
    g.path = packed_ok ? (opts.path == 3 ? 3 : 2) : 1;
    if (g.path >= 2) {
        g.nf = nf_packed;
        g.width = w_packed;
        const double sigma = (double)g.nf / (double)g.I;
        g.beta = 0.97 * kPi * (1.0 - 0.5 / sigma) * g.width;
    } else {
        g.nf = std::max<int64_t>(64, next_pow2((int64_t)std::ceil(std::max(2.0, opts.sigma) * (double)g.I)));
        g.width = std::min(16, std::max(2, (int)std::ceil(std::log10(1.0 / p->tol)) + 1));
        g.beta = 2.30 * g.width;
    }
    g.log_nf = ilog2(g.nf);                      // ceil(log2 nf)
    const double s_cells = (double)g.nf * g.df;  // cells per unit time
    g.h = 1.0 / s_cells;
    const double span_cells = (ts.back() - ts.front()) * s_cells;
    g.wrap = (span_cells + g.width + 2.0 >= (double)g.nf) ? 1 : 0;
    const double half_w = 0.5 * g.width;
    g.t_ref = g.wrap ? ts.front() : ts.front() - half_w * g.h;

    struct Pt {
        int64_t cell;
        double off;
        int64_t src;    // caller index
        int64_t sidx;   // sorted index
        double uh;
    };
    std::vector<Pt> pts(N);
    const double nf_d = (double)g.nf;
    for (int64_t j = 0; j < N; ++j) {
        const double d = ts[j] - g.t_ref;
        double uh, ul;
        two_prod(d, s_cells, uh, ul);
        if (g.wrap) uh -= std::floor(uh / nf_d) * nf_d;  // exact: the result is a multiple of ulp(uh)
        const int64_t i0 = (int64_t)std::ceil(uh - half_w);
        const double off = ((double)i0 - uh) - ul;
        pts[j] = {i0, off, ord[j], j, uh};
    }
    if (g.wrap) {
        std::stable_sort(pts.begin(), pts.end(), [](const Pt& a, const Pt& b) {
            return a.cell < b.cell || (a.cell == b.cell && a.uh < b.uh);
        });
        std::vector<Pt> ext;
        for (const Pt& q : pts)
            if (q.cell + g.width > g.nf) {
                Pt c = q;
                c.cell -= g.nf;
                ext.push_back(c);
            }
        for (const Pt& q : pts) ext.push_back(q);
        for (const Pt& q : pts)
            if (q.cell < 0) {
                Pt c = q;
                c.cell += g.nf;
                ext.push_back(c);
            }
        pts.swap(ext);
    }
    // ---- exec path and the nf = n1 * n2 split ----
    // rows(n2): nonzero input rows of the column DFTs for a row length n2
    const int64_t last_cell = g.wrap ? g.nf : pts.back().cell + g.width;  // one past the last written cell
    auto rows_for = [&](int64_t n2) {
        const int64_t n1 = g.nf / n2;
        return g.wrap ? n1 : std::min<int64_t>(n1, (last_cell + n2 - 1) / n2);
    };
    if (g.path >= 2) {
        g.n2 = 1024;
        g.n1 = g.nf / 1024;
        g.log_n2 = 10;
        g.log_n1 = ilog2(g.n1);  // not used by the packed kernels (n1 = 2^a or 3 * 2^a)
    } else {
        g.log_n1 = g.log_nf / 2;
        g.log_n2 = g.log_nf - g.log_n1;
        g.n1 = int64_t(1) << g.log_n1;
        g.n2 = int64_t(1) << g.log_n2;
    }
    g.rows = rows_for(g.n2);
    if (g.path >= 2 && g.rows > 64) {
        set_error("internal: packed path support exceeds 64 rows");
        return bail(M2_ERR_ARG);
    }
    g.kp = g.path >= 2 ? (K + 1) / 2 : K;
    g.Lg = g.rows * g.n2;
    g.P = (int64_t)pts.size();
    g.ntiles = (g.Lg + kSpreadTile - 1) / kSpreadTile;
    // CTA shapes of the FFT passes: at most 8192 (FP32) / 4096 (FP64) complex values in shared memory
    const int64_t ecta = opts.precision == 32 ? 8192 : 4096;
    g.cw = (int)std::max<int64_t>(1, std::min<int64_t>(g.n2, ecta / g.n1));
    g.rw = (int)std::max<int64_t>(1, std::min<int64_t>(g.n1, ecta / g.n2));
    // small transforms: fewer columns / rows per CTA until one signal's pass has two CTAs per SM
    // (each column and row is transformed on its own, so the shape does not change the result)
    while (g.cw > 1 && (g.n2 / g.cw) * (int64_t)K < 2 * (int64_t)p->sm_count) g.cw /= 2;
    while (g.rw > 1 && (g.n1 / g.rw) < 2 * (int64_t)p->sm_count) g.rw /= 2;
    const size_t csz = opts.precision == 32 ? 8 : 16;
    {
        // generic path: keep a chunk's workspace within L2.  Packed four-kernel path: 4 to 16
        // signals, 64 MiB / (2 * K/2 * nf complex) per signal -- consecutive chunks run overlapped
        // on two streams, so smaller chunks keep more of both in L2, while below 4 the grids get
        // too small (measured on GB300: 4 is best for I = 2^18, within 1 % of best for I = 2^20).
        // The persistent kernel: up to 16 (its ring of workspace slots).
        const size_t z_per_signal = (size_t)g.kp * g.nf * csz * (g.path >= 2 ? 2 : 1);
        int64_t chunk;
        if (g.path == 2) {
            chunk = std::max<int64_t>(4, std::min<int64_t>(16, (int64_t)((size_t(64) << 20) / z_per_signal)));
        } else if (g.path == 3) {
            chunk = std::max<int64_t>(1, std::min<int64_t>(16, (int64_t)((size_t(1) << 30) / z_per_signal)));
        } else {
            chunk = std::max<int64_t>(1, (int64_t)((48u << 20) / std::max<size_t>(z_per_signal, 1)));
            chunk = std::min<int64_t>(chunk, 1024);
        }
        if (opts.max_batch > 0)  // packed paths: the chunk asked for (at most 64); generic: a cap
            chunk = g.path >= 2 ? std::min<int64_t>(opts.max_batch, 64) : std::min<int64_t>(chunk, opts.max_batch);
        g.chunk = (int)chunk;
    }
    g.twb_bits = (g.log_nf + 1) / 2;

    // ---- point arrays ----
    {
        std::vector<int32_t> src(g.P), cell(g.P);
        std::vector<double> off(g.P);
        for (int64_t q = 0; q < g.P; ++q) {
            src[q] = (int32_t)pts[q].src;
            cell[q] = (int32_t)pts[q].cell;
            off[q] = pts[q].off;
        }
        M2_TRY_OR(pb.upload(&p->d_pt_src, src));
        M2_TRY_OR(pb.upload(&p->d_pt_cell, cell));
        if (opts.precision == 32) M2_TRY_OR(upload_typed<float>(pb, &p->d_pt_off, off));
        else M2_TRY_OR(upload_typed<double>(pb, &p->d_pt_off, off));

        // modulated tapers u_k(t_n) = w_k(t_n) exp(-i 2 pi f_mid t_n)
        std::vector<double> tap;
        if (g.real_taper) {
            tap.resize((size_t)K * g.P);
            for (int k = 0; k < K; ++k)
                for (int64_t q = 0; q < g.P; ++q) tap[(size_t)k * g.P + q] = w_sorted[(size_t)k * N + pts[q].sidx];
        } else {
            tap.resize((size_t)2 * K * g.P);
            for (int64_t q = 0; q < g.P; ++q) {
                const double cyc = frac_cycles(g.fmid_hi, g.fmid_lo, ts[pts[q].sidx]);
                const double c = std::cos(2.0 * kPi * cyc), s = std::sin(2.0 * kPi * cyc);
                for (int k = 0; k < K; ++k) {
                    // conj(w_k) e^{-i 2 pi f_mid t} (Eq. eigencoefficients: the conjugated taper)
                    const double wv = w_sorted[(size_t)k * N + pts[q].sidx];
                    const double wi = cplx ? w_sorted_im[(size_t)k * N + pts[q].sidx] : 0.0;
                    tap[2 * ((size_t)k * g.P + q)] = wv * c - wi * s;
                    tap[2 * ((size_t)k * g.P + q) + 1] = -wv * s - wi * c;
                }
            }
        }
        if (opts.precision == 32) M2_TRY_OR(upload_typed<float>(pb, &p->d_taper, tap));
        else M2_TRY_OR(upload_typed<double>(pb, &p->d_taper, tap));

        // spreading tiles: points whose window [cell, cell + w) meets [c0, c1)
        std::vector<int32_t> tpb(g.ntiles), tpe(g.ntiles);
        for (int64_t j = 0; j < g.ntiles; ++j) {
            const int64_t c0 = j * kSpreadTile, c1 = std::min<int64_t>(c0 + kSpreadTile, g.Lg);
            auto lo = std::lower_bound(cell.begin(), cell.end(), (int32_t)(c0 - g.width + 1));
            auto hi = std::lower_bound(cell.begin(), cell.end(), (int32_t)c1);
            tpb[j] = (int32_t)(lo - cell.begin());
            tpe[j] = (int32_t)(hi - cell.begin());
        }
        M2_TRY_OR(pb.upload(&p->d_tile_pb, tpb));
        M2_TRY_OR(pb.upload(&p->d_tile_pe, tpe));

        if (g.path >= 2) {
            // cell-major spreading matrix (sliced ELL, slices of 32 cells): entry e of cell c is the
            // e-th point p (ascending) whose window covers c, with the window value phi(c - u_p)
            // evaluated in FP64 and rounded once to FP32; every cell of a slice has the slice's
            // largest count of entries (padding entries are skipped)
            const int Kp = (K + 1) / 2;
            const int64_t nsl = (g.Lg + 31) / 32;
            const int spt = kSpreadTile / 32;  // slices per tile
            std::vector<int32_t> cnt((size_t)g.Lg, 0);
            for (int64_t q = 0; q < g.P; ++q)
                for (int d = 0; d < g.width; ++d) {
                    const int64_t cc = (int64_t)cell[q] + d;
                    if (cc >= 0 && cc < g.Lg) ++cnt[(size_t)cc];
                }
            std::vector<int2> sl((size_t)nsl);
            int64_t ne = 0;
            for (int64_t s = 0; s < nsl; ++s) {
                int e = 0;
                for (int64_t cc = 32 * s; cc < std::min<int64_t>(32 * s + 32, g.Lg); ++cc) e = std::max(e, cnt[(size_t)cc]);
                sl[(size_t)s] = make_int2((int)ne, e);
                ne += 32 * (int64_t)e;
                if (ne > (int64_t)INT32_MAX) {
                    set_error("internal: spreading matrix exceeds 2^31 entries");
                    return bail(M2_ERR_ARG);
                }
            }
            std::vector<int32_t> ep((size_t)ne, -1);  // point of each entry (-1: padding)
            std::vector<float> ephi((size_t)ne, 0.f);
            std::fill(cnt.begin(), cnt.end(), 0);  // now the fill cursor of each cell
            const double two_over_w = 2.0 / g.width;
            for (int64_t q = 0; q < g.P; ++q)
                for (int d = 0; d < g.width; ++d) {
                    const int64_t cc = (int64_t)cell[q] + d;
                    if (cc < 0 || cc >= g.Lg) continue;
                    const int64_t idx = sl[(size_t)(cc >> 5)].x + 32 * (int64_t)cnt[(size_t)cc]++ + (cc & 31);
                    ep[(size_t)idx] = (int32_t)q;
                    const double a = (off[q] + (double)d) * two_over_w;
                    ephi[(size_t)idx] = (float)std::exp(g.beta * (std::sqrt(std::max(0.0, 1.0 - a * a)) - 1.0));
                }
            // per tile: its entries (contiguous: its slices), its points (contiguous: points are in
            // cell order) and the run of samples they read; staged in shared memory when the run
            // spans at most kMaxStagedRun samples and the caps of all staged tiles fit the budget
            constexpr int kMaxStagedRun = 1024;
            constexpr size_t kStageBudget = size_t(96) << 10;  // at 4 signals per CTA
            std::vector<int4> tb((size_t)g.ntiles), tr((size_t)g.ntiles);
            std::vector<char> staged((size_t)g.ntiles, 0);
            for (int64_t t = 0; t < g.ntiles; ++t) {
                const int64_t s0 = t * spt, s1 = std::min<int64_t>(s0 + spt, nsl);
                const int64_t e0 = sl[(size_t)s0].x, e1 = s1 < nsl ? sl[(size_t)s1].x : ne;
                int pmin = INT32_MAX, pmax = -1;
                for (int64_t e = e0; e < e1; ++e)
                    if (ep[(size_t)e] >= 0) {
                        pmin = std::min(pmin, ep[(size_t)e]);
                        pmax = std::max(pmax, ep[(size_t)e]);
                    }
                int smin = INT32_MAX, smax = -1;
                for (int q = pmin; q <= pmax && pmax >= 0; ++q) {
                    smin = std::min(smin, src[q]);
                    smax = std::max(smax, src[q]);
                }
                const int np = pmax >= 0 ? pmax - pmin + 1 : 0;
                const int run = smax >= smin ? smax - smin + 1 : 0;
                tb[(size_t)t] = make_int4((int)e0, (int)(e1 - e0), np > 0 ? pmin : 0, np);
                tr[(size_t)t] = make_int4(run > 0 ? smin : 0, run, 0, 0);
                staged[(size_t)t] = np > 0 && np <= 65535 && run <= kMaxStagedRun;
            }
            int ecap = 0, pcap = 0, ncap = 0;
            for (;;) {
                ecap = pcap = ncap = 0;
                int64_t big = -1;
                for (int64_t t = 0; t < g.ntiles; ++t)
                    if (staged[(size_t)t]) {
                        ecap = std::max(ecap, (tb[(size_t)t].y + 3) & ~3);
                        pcap = std::max(pcap, (tb[(size_t)t].w + 3) & ~3);
                        ncap = std::max(ncap, (tr[(size_t)t].y + 3) & ~3);
                        if (big < 0 || tb[(size_t)t].y > tb[(size_t)big].y) big = t;
                    }
                if (big < 0 || packed::spread_ell_smem_bytes(Kp, 4, ecap, pcap, ncap) <= kStageBudget) break;
                staged[(size_t)big] = 0;
            }
            std::vector<uint2> ee((size_t)ne);
            for (int64_t t = 0; t < g.ntiles; ++t) {
                tr[(size_t)t].z = staged[(size_t)t] ? 1 : 0;
                for (int64_t e = tb[(size_t)t].x; e < (int64_t)tb[(size_t)t].x + tb[(size_t)t].y; ++e) {
                    const int q = ep[(size_t)e];
                    uint32_t word = 0xffffffffu;
                    if (q >= 0)
                        word = staged[(size_t)t] ? (uint32_t)(q - tb[(size_t)t].z) |
                                                       ((uint32_t)(src[q] - tr[(size_t)t].x) << 16)
                                                 : (uint32_t)q;
                    uint32_t phib;
                    std::memcpy(&phib, &ephi[(size_t)e], 4);
                    ee[(size_t)e] = make_uint2(word, phib);
                }
            }
            // taper pairs point-major: tap2[q][j] = (u_{2j}[q], u_{2j+1}[q]) (u_K = 0 for odd K)
            std::vector<float> t2((size_t)g.P * 2 * Kp, 0.f);
            for (int64_t q = 0; q < g.P; ++q)
                for (int k = 0; k < K; ++k) t2[(size_t)q * 2 * Kp + k] = (float)tap[(size_t)k * g.P + q];
            M2_TRY_OR(pb.upload(&p->d_ell_slice, sl));
            M2_TRY_OR(pb.upload(&p->d_ell_e, ee));
            M2_TRY_OR(pb.upload(&p->d_ell_tile, tb));
            M2_TRY_OR(pb.upload(&p->d_ell_run, tr));
            M2_TRY_OR(pb.upload(&p->d_tap2, t2));
            p->ell_ecap = ecap;
            p->ell_pcap = pcap;
            p->ell_ncap = ncap;
            p->ell_entries = ne;
        }
    }

    // ---- twiddles ----
    M2_TRY_OR(upload_complex(pb, p->precision, &p->d_tw1, unit_roots(g.n1 / 2, g.n1, 1)));
    M2_TRY_OR(upload_complex(pb, p->precision, &p->d_tw2, unit_roots(g.n2 / 2, g.n2, 1)));
    M2_TRY_OR(upload_complex(pb, p->precision, &p->d_twa,
                             unit_roots((g.nf + (int64_t(1) << g.twb_bits) - 1) >> g.twb_bits, g.nf,
                                        int64_t(1) << g.twb_bits)));
    M2_TRY_OR(upload_complex(pb, p->precision, &p->d_twb, unit_roots(int64_t(1) << g.twb_bits, g.nf, 1)));
    if (g.path >= 2) {
        M2_TRY_OR(upload_complex(pb, p->precision, &p->d_twn1, unit_roots(g.n1, g.n1, 1)));
        {
            // row-FFT twiddles in the order a warp reads them: [cc][lane] = W_1024^{cc lane}
            std::vector<double> t32(2 * 1024);
            for (int cc = 0; cc < 32; ++cc) {
                const std::vector<double> r = unit_roots(32, 1024, cc);
                std::copy(r.begin(), r.end(), t32.begin() + 64 * cc);
            }
            M2_TRY_OR(upload_complex(pb, p->precision, &p->d_tw1024, t32));
        }
        M2_CUDA_TRY_OR(cudaHostAlloc(reinterpret_cast<void**>(&p->stage_status), 4 * sizeof(int), cudaHostAllocMapped));
        std::memset(p->stage_status, 0, 4 * sizeof(int));
        M2_CUDA_TRY_OR(cudaHostGetDevicePointer(reinterpret_cast<void**>(&p->d_stage_status), p->stage_status, 0));
        int64_t F = 1;
        while (F < 32 && g.n1 % (F * 2) == 0) F *= 2;
        g.colF = (int)F;
        const int64_t C = g.n1 / F;
        // colT[q][l2] = W_nf^{l2 C q}, colB[r][l2] = W_nf^{l2 r}
        std::vector<double> tT(2 * F * 1024), tB(2 * C * 1024);
        for (int64_t q = 0; q < F; ++q)
            for (int64_t l2 = 0; l2 < 1024; ++l2) {
                const int64_t e = (l2 * C * q) % g.nf;
                const double x = 2.0 * (double)e / (double)g.nf;
                tT[2 * (q * 1024 + l2)] = std::cos(kPi * x);
                tT[2 * (q * 1024 + l2) + 1] = -std::sin(kPi * x);
            }
        for (int64_t r = 0; r < C; ++r)
            for (int64_t l2 = 0; l2 < 1024; ++l2) {
                const int64_t e = (l2 * r) % g.nf;
                const double x = 2.0 * (double)e / (double)g.nf;
                tB[2 * (r * 1024 + l2)] = std::cos(kPi * x);
                tB[2 * (r * 1024 + l2) + 1] = -std::sin(kPi * x);
            }
        M2_TRY_OR(upload_complex(pb, p->precision, &p->d_colT, tT));
        M2_TRY_OR(upload_complex(pb, p->precision, &p->d_colB, tB));
        // fold twiddles of the column pass: colFw[r][l1] = W_n1^{(l1 r) mod n1}, the entries of the
        // [n1] table that coset r reads for input row l1
        const std::vector<double> tn1 = unit_roots(g.n1, g.n1, 1);
        std::vector<double> tF(2 * C * g.rows);
        for (int64_t r = 0; r < C; ++r)
            for (int64_t l1 = 0; l1 < g.rows; ++l1) {
                const int64_t e = (l1 * r) % g.n1;
                tF[2 * (r * g.rows + l1)] = tn1[2 * e];
                tF[2 * (r * g.rows + l1) + 1] = tn1[2 * e + 1];
            }
        M2_TRY_OR(upload_complex(pb, p->precision, &p->d_colFw, tF));
    }

    // ---- deconvolution / re-phasing factors ----
    {
        const int Q = 200;
        std::vector<double> gx, gw;
        gauss_legendre(Q, gx, gw);
        std::vector<double> zq(Q), pw(Q);
        for (int q = 0; q < Q; ++q) {
            const double z = 0.25 * g.width * (gx[q] + 1.0);  // [0, w/2]
            const double a = 2.0 * z / g.width;
            const double phi = std::exp(g.beta * (std::sqrt(std::max(0.0, 1.0 - a * a)) - 1.0));
            zq[q] = z;
            pw[q] = 0.25 * g.width * gw[q] * phi;
        }
        double *dz = nullptr, *dpw = nullptr;
        M2_CUDA_TRY_OR(cudaMalloc(&dz, Q * sizeof(double)));
        M2_CUDA_TRY_OR(cudaMalloc(&dpw, Q * sizeof(double)));
        cudaMemcpy(dz, zq.data(), Q * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(dpw, pw.data(), Q * sizeof(double), cudaMemcpyHostToDevice);
        double ah, al;
        two_prod(g.df, g.t_ref, ah, al);
        const unsigned blocks = (unsigned)((g.I + 255) / 256);
        if (p->precision == 32) {
            float2* d = nullptr;
            M2_TRY_OR(pb.alloc(&d, g.I));
            deconv_kernel<float2><<<blocks, 256>>>(g.I, g.i_c, 1.0 / nf_d, dz, dpw, Q, ah, al, d);
            p->d_deconv = d;
        } else {
            double2* d = nullptr;
            M2_TRY_OR(pb.alloc(&d, g.I));
            deconv_kernel<double2><<<blocks, 256>>>(g.I, g.i_c, 1.0 / nf_d, dz, dpw, Q, ah, al, d);
            p->d_deconv = d;
        }
        cudaError_t e = cudaDeviceSynchronize();
        cudaFree(dz);
        cudaFree(dpw);
        if (e != cudaSuccess) {
            set_error("deconvolution kernel failed: %s", cudaGetErrorString(e));
            return bail(M2_ERR_CUDA);
        }
    }

    // ---- taper sums W_k^0(0) = sum_n w_k(t_n) for the F-statistic (Sec. 3, Eq. f_stat) ----
    {
        std::vector<double> ws(K, 0.0);
        double q = 0.0;
        for (int k = 0; k < K; ++k) {
            for (int64_t j = 0; j < N; ++j) ws[k] += w_sorted[(size_t)k * N + j];
            q += ws[k] * ws[k];
        }
        p->wq = q;
        if (opts.precision == 32) M2_TRY_OR(upload_typed<float>(pb, &p->d_wsum, ws));
        else M2_TRY_OR(upload_typed<double>(pb, &p->d_wsum, ws));
    }

    // ---- leakage estimate (App. B) ----
    M2_TRY_OR(pb.alloc(&p->d_Lhat, (size_t)K * g.I));
    M2_TRY_OR(pb.alloc(&p->d_Ehat, (size_t)g.I));
    if (p->have_lambda && !cplx) {
        const unsigned blocks = (unsigned)((g.I + 127) / 128);
        if (integer_grid) {
            std::vector<double> Lk(K);
            for (int k = 0; k < K; ++k) {
                double nrm = 0;
                for (int64_t j = 0; j < N; ++j) nrm += w_sorted[(size_t)k * N + j] * w_sorted[(size_t)k * N + j];
                Lk[k] = std::fabs(p->lambda[k] - p->lambda[k] * 2.0 * f_w / nrm);
            }
            double* dLk = nullptr;
            M2_CUDA_TRY_OR(cudaMalloc(&dLk, K * sizeof(double)));
            cudaMemcpy(dLk, Lk.data(), K * sizeof(double), cudaMemcpyHostToDevice);
            leakage_const_kernel<<<blocks, 128>>>(K, g.I, dLk, p->d_Lhat, p->d_Ehat);
            cudaError_t e = cudaDeviceSynchronize();
            cudaFree(dLk);
            if (e != cudaSuccess) {
                set_error("leakage kernel failed: %s", cudaGetErrorString(e));
                return bail(M2_ERR_CUDA);
            }
            p->have_leakage = 1;
        } else if ((double)N * (double)N * (double)g.I <= 1.0e9) {
            double tbar = 0;
            for (double v : ts) tbar += v;
            tbar /= (double)N;
            std::vector<double> tc(N);
            for (int64_t j = 0; j < N; ++j) tc[j] = ts[j] - tbar;
            double *dtc = nullptr, *dw = nullptr, *dl = nullptr;
            M2_CUDA_TRY_OR(cudaMalloc(&dtc, N * sizeof(double)));
            M2_CUDA_TRY_OR(cudaMalloc(&dw, (size_t)K * N * sizeof(double)));
            M2_CUDA_TRY_OR(cudaMalloc(&dl, K * sizeof(double)));
            cudaMemcpy(dtc, tc.data(), N * sizeof(double), cudaMemcpyHostToDevice);
            cudaMemcpy(dw, w_sorted.data(), (size_t)K * N * sizeof(double), cudaMemcpyHostToDevice);
            cudaMemcpy(dl, p->lambda.data(), K * sizeof(double), cudaMemcpyHostToDevice);
            leakage_direct_kernel<<<(unsigned)g.I, kLeakThreads>>>((int)N, K, g.I, dtc, dw, fmax, g.f_lo, g.df,
                                                                    dl, f_w, p->d_Lhat, p->d_Ehat);
            cudaError_t e = cudaDeviceSynchronize();
            cudaFree(dtc);
            cudaFree(dw);
            cudaFree(dl);
            if (e != cudaSuccess) {
                set_error("leakage kernel failed: %s", cudaGetErrorString(e));
                return bail(M2_ERR_CUDA);
            }
            p->have_leakage = 1;
        } else {
            M2_TRY_OR(windowed_leakage(p, ts));
            p->have_leakage = 1;
        }
    } else if (p->have_lambda && cplx && (double)N * (double)N * (double)g.I <= 1.0e9) {
        // sub-band plan: the direct pair sum with R(B^q) and the shifts from the nominal centre
        double tbar = 0;
        for (double v : ts) tbar += v;
        tbar /= (double)N;
        std::vector<double> tc(N);
        for (int64_t j = 0; j < N; ++j) tc[j] = ts[j] - tbar;
        double *dtc = nullptr, *dwr = nullptr, *dwi = nullptr, *dl = nullptr;
        M2_CUDA_TRY_OR(cudaMalloc(&dtc, N * sizeof(double)));
        M2_CUDA_TRY_OR(cudaMalloc(&dwr, (size_t)K * N * sizeof(double)));
        M2_CUDA_TRY_OR(cudaMalloc(&dwi, (size_t)K * N * sizeof(double)));
        M2_CUDA_TRY_OR(cudaMalloc(&dl, K * sizeof(double)));
        cudaMemcpy(dtc, tc.data(), N * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(dwr, w_sorted.data(), (size_t)K * N * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(dwi, w_sorted_im.data(), (size_t)K * N * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(dl, p->lambda.data(), K * sizeof(double), cudaMemcpyHostToDevice);
        leakage_direct_cplx_kernel<<<(unsigned)g.I, kLeakThreadsC>>>((int)N, K, g.I, dtc, dwr, dwi, sb->f_min,
                                                                      sb->f_max, g.f_lo, g.df, dl, f_w, p->d_Lhat,
                                                                      p->d_Ehat);
        cudaError_t e = cudaDeviceSynchronize();
        cudaFree(dtc);
        cudaFree(dwr);
        cudaFree(dwi);
        cudaFree(dl);
        if (e != cudaSuccess) {
            set_error("leakage kernel failed: %s", cudaGetErrorString(e));
            return bail(M2_ERR_CUDA);
        }
        p->have_leakage = 1;
    }

    // ---- workspace ----
    if (opts.precision == 32) {
        float2 *dg = nullptr, *dZ = nullptr;
        M2_TRY_OR(pb.alloc(&dg, (size_t)g.chunk * g.kp * g.Lg));
        M2_TRY_OR(pb.alloc(&dZ, (size_t)g.chunk * g.kp * g.nf));
        p->d_g = dg;
        p->d_Z = dZ;
    } else {
        double2 *dg = nullptr, *dZ = nullptr;
        M2_TRY_OR(pb.alloc(&dg, (size_t)g.chunk * g.kp * g.Lg));
        M2_TRY_OR(pb.alloc(&dZ, (size_t)g.chunk * g.kp * g.nf));
        p->d_g = dg;
        p->d_Z = dZ;
    }
    M2_CUDA_TRY_OR(cudaDeviceSynchronize());
    *out = p;
    return M2_OK;
}

// Time `reps` execs of B synthetic signals on plan p (ms per exec, the fastest repetition).
m2_status time_exec(m2nufft_plan_t p, int64_t B, int reps, double* ms) {
    const Geometry& g = p->g;
    const size_t nx = (size_t)B * g.N, nj = (size_t)B * g.K * g.I, np = (size_t)B * g.I;
    float *x = nullptr, *E = nullptr, *P = nullptr;
    float2* J = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    m2_status rs = M2_OK;
    cudaError_t e = cudaMalloc(&x, sizeof(float) * nx);
    if (e == cudaSuccess) e = cudaMalloc(&J, sizeof(float2) * nj);
    if (e == cudaSuccess) e = cudaMalloc(&E, sizeof(float) * nj);
    if (e == cudaSuccess) e = cudaMalloc(&P, sizeof(float) * np);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        std::vector<float> hx(nx);
        uint64_t z = 0x9e3779b97f4a7c15ull;  // any signal does: the work does not depend on x
        for (size_t i = 0; i < nx; ++i) {
            z ^= z << 13;
            z ^= z >> 7;
            z ^= z << 17;
            hx[i] = (float)((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
        }
        e = cudaMemcpy(x, hx.data(), sizeof(float) * nx, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        set_error("autotune: %s", cudaGetErrorString(e));
        rs = e == cudaErrorMemoryAllocation ? M2_ERR_NOMEM : M2_ERR_CUDA;
    }
    double best = 1e300;
    for (int r = -2; r < reps && rs == M2_OK; ++r) {  // two untimed warm-up execs
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) rs = m2nufft_exec(p, x, B, J, E, P, nullptr, nullptr, st);
        if (rs == M2_OK && (e = cudaEventRecord(e1, st)) == cudaSuccess) e = cudaEventSynchronize(e1);
        float tm = 0.f;
        if (rs == M2_OK && e == cudaSuccess) e = cudaEventElapsedTime(&tm, e0, e1);
        if (rs == M2_OK && e != cudaSuccess) {
            set_error("autotune: %s", cudaGetErrorString(e));
            rs = M2_ERR_CUDA;
        }
        if (r >= 0) best = std::min(best, (double)tm);
    }
    if (st) cudaStreamSynchronize(st);
    cudaFree(x);
    cudaFree(J);
    cudaFree(E);
    cudaFree(P);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    *ms = best;
    return rs;
}

// Autotuning (m2_opts.tune = 1): the default plan, then candidates built from its tapers --
// sigma 2, chunks of 4, 8 and 16 signals (those other than the default), the persistent path --
// each timed on a synthetic batch of 32 signals; the fastest configuration is rebuilt with the plan's eigenvalues
// (for the leakage estimate) and returned.  Plans that take the generic path are returned untuned.
m2_status tuned_plan(const double* t, int64_t N, double fs, double f_w, int K, const m2_fgrid* fc,
                     const double* w_given, const double* lam_given, const m2_opts* opts_in, m2nufft_plan_t* out) {
    m2_opts base = *opts_in;
    base.tune = 0;
    m2nufft_plan_t p0 = nullptr;
    M2_TRY(build_plan(t, N, fs, f_w, K, fc, w_given, lam_given, &base, &p0));
    if (p0->g.path < 2) {
        *out = p0;
        return M2_OK;
    }
    DeviceGuard guard(p0->device);
    const std::vector<double> w = p0->w;
    const std::vector<double> lam = p0->lambda;
    const bool have_lam = p0->have_lambda != 0;
    const int64_t B = 32;  // two chunks of the largest candidate
    std::vector<m2_opts> cand;
    m2_opts c = base;
    c.path = 2;
    cand.push_back(c);  // the default configuration (p0)
    c.sigma = 2.0;
    cand.push_back(c);
    for (int ch : {4, 8, 16}) {
        if (ch == p0->g.chunk) continue;
        c = base;
        c.path = 2;
        c.max_batch = ch;
        cand.push_back(c);
    }
    c = base;
    c.path = 3;
    cand.push_back(c);
    std::vector<double> ms(cand.size(), 1e300);
    m2_status st = time_exec(p0, B, 3, &ms[0]);
    for (size_t i = 1; i < cand.size() && st == M2_OK; ++i) {
        m2nufft_plan_t pc = nullptr;
        m2_status s2 = build_plan(t, N, fs, f_w, K, fc, w.data(), nullptr, &cand[i], &pc);
        if (s2 != M2_OK) {  // a candidate the pattern does not admit (e.g. sigma 2 beyond the packed limits)
            clear_error();
            continue;
        }
        st = time_exec(pc, B, 3, &ms[i]);
        free_plan(pc);
    }
    if (st != M2_OK) {
        free_plan(p0);
        return st;
    }
    size_t best = 0;
    for (size_t i = 1; i < cand.size(); ++i)
        if (ms[i] < ms[best]) best = i;
    m2nufft_plan_t pf = p0;
    if (best != 0) {
        free_plan(p0);
        st = build_plan(t, N, fs, f_w, K, fc, w.data(), have_lam ? lam.data() : nullptr, &cand[best], &pf);
        if (st != M2_OK) return st;
    }
    pf->tune_opts = cand;
    pf->tune_ms = ms;
    *out = pf;
    return M2_OK;
}

}  // namespace
}  // namespace m2

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" m2_status m2nufft_plan(const double* t, int64_t N, double fs, double f_w, int K, const m2_fgrid* fc,
                                  const m2_opts* opts, m2nufft_plan_t* out) {
    m2::clear_error();
    if (opts && opts->tune) return m2::tuned_plan(t, N, fs, f_w, K, fc, nullptr, nullptr, opts, out);
    return m2::build_plan(t, N, fs, f_w, K, fc, nullptr, nullptr, opts, out);
}

extern "C" m2_status m2nufft_get_tuning(m2nufft_plan_t p, int* n, m2_opts* opts, double* ms) {
    m2::clear_error();
    if (!p || !n) {
        m2::set_error("plan or n is NULL");
        return M2_ERR_ARG;
    }
    *n = (int)p->tune_ms.size();
    for (size_t i = 0; i < p->tune_ms.size(); ++i) {
        if (opts) opts[i] = p->tune_opts[i];
        if (ms) ms[i] = p->tune_ms[i];
    }
    return M2_OK;
}

extern "C" m2_status m2nufft_plan_with_tapers(const double* t, int64_t N, double fs, double f_w, int K,
                                              const m2_fgrid* fc, const double* w, const double* lambda,
                                              const m2_opts* opts, m2nufft_plan_t* out) {
    m2::clear_error();
    if (!w) {
        m2::set_error("w is NULL");
        return M2_ERR_ARG;
    }
    if (opts && opts->tune) return m2::tuned_plan(t, N, fs, f_w, K, fc, w, lambda, opts, out);
    return m2::build_plan(t, N, fs, f_w, K, fc, w, lambda, opts, out);
}

extern "C" m2_status m2nufft_plan_subband(const double* t, int64_t N, double fs, double f_w, int K,
                                          const m2_subband* sb, const m2_fgrid* fc, const double* w,
                                          const double* lambda, const m2_opts* opts, m2nufft_plan_t* out) {
    m2::clear_error();
    if (!sb) {
        m2::set_error("sub-band is NULL");
        return M2_ERR_ARG;
    }
    return m2::build_plan(t, N, fs, f_w, K, fc, nullptr, lambda, opts, out, sb, w);
}

extern "C" m2_status m2nufft_get_tapers_complex(m2nufft_plan_t p, double* w, double* lambda) {
    m2::clear_error();
    if (!p) {
        m2::set_error("plan is NULL");
        return M2_ERR_ARG;
    }
    if (w) {
        for (size_t q = 0; q < p->w.size(); ++q) {
            w[2 * q] = p->w[q];
            w[2 * q + 1] = p->complex_taper ? p->w_im[q] : 0.0;
        }
    }
    if (lambda) {
        if (p->have_lambda) std::memcpy(lambda, p->lambda.data(), sizeof(double) * p->lambda.size());
        else
            for (int k = 0; k < p->g.K; ++k) lambda[k] = std::nan("");
    }
    return M2_OK;
}

extern "C" m2_status m2nufft_get_tapers(m2nufft_plan_t p, double* w, double* lambda) {
    m2::clear_error();
    if (!p) {
        m2::set_error("plan is NULL");
        return M2_ERR_ARG;
    }
    if (w && p->complex_taper) {
        m2::set_error("m2nufft_get_tapers: the plan's tapers are complex; use m2nufft_get_tapers_complex");
        return M2_ERR_ARG;
    }
    if (w) std::memcpy(w, p->w.data(), sizeof(double) * p->w.size());
    if (lambda) {
        if (p->have_lambda) std::memcpy(lambda, p->lambda.data(), sizeof(double) * p->lambda.size());
        else
            for (int k = 0; k < p->g.K; ++k) lambda[k] = std::nan("");
    }
    return M2_OK;
}

extern "C" m2_status m2nufft_get_leakage(m2nufft_plan_t p, double* Lhat, double* Ehat) {
    m2::clear_error();
    if (!p) {
        m2::set_error("plan is NULL");
        return M2_ERR_ARG;
    }
    if ((Lhat || Ehat) && !p->have_leakage) {
        m2::set_error("leakage estimate not available for this plan");
        return M2_ERR_ARG;
    }
    m2::DeviceGuard guard(p->device);
    if (Lhat) M2_CUDA_TRY(cudaMemcpy(Lhat, p->d_Lhat, sizeof(double) * p->g.K * p->g.I, cudaMemcpyDeviceToHost));
    if (Ehat) M2_CUDA_TRY(cudaMemcpy(Ehat, p->d_Ehat, sizeof(double) * p->g.I, cudaMemcpyDeviceToHost));
    return M2_OK;
}

extern "C" m2_status m2nufft_get_info(m2nufft_plan_t p, m2_info* info) {
    m2::clear_error();
    if (!p || !info) {
        m2::set_error("plan or info is NULL");
        return M2_ERR_ARG;
    }
    const m2::Geometry& g = p->g;
    info->N = g.N;
    info->K = g.K;
    info->I = g.I;
    info->precision = p->precision;
    info->width = g.width;
    info->beta = g.beta;
    info->nf = g.nf;
    info->n1 = g.n1;
    info->n2 = g.n2;
    info->rows = g.rows;
    info->wrap = g.wrap;
    info->real_taper = g.real_taper;
    info->integer_grid = p->integer_grid;
    info->chunk = g.chunk;
    info->path = g.path;
    info->device_bytes = p->device_bytes;
    info->gep_seconds = p->gep_seconds;
    info->spread_entries = p->ell_entries;
    return M2_OK;
}

extern "C" m2_status m2nufft_destroy(m2nufft_plan_t p) {
    m2::clear_error();
    m2::free_plan(p);
    return M2_OK;
}

extern "C" const char* m2nufft_last_error(void) { return m2::g_last_error.c_str(); }

extern "C" const char* m2nufft_version(void) { return "m2nufft-gb300 0.1 (sm_103a)"; }
