// The suboptimality measure with the optimal per-band eigenvalues (Sec. 3,
// Eq. subopt_measure):  E_i = (1/K) sum_k |lambda_k^i - lambda_k^0|,
// where lambda_k^i are the K largest eigenvalues of the GEP at band A_i,
//   R(A_i) w = lambda R(B) w,  R(A_i) = D_i R(A0) D_i^*,  D_i = diag(e^{i 2 pi f_i t_n})
// (Eq. gpss_matrix_a centred at f_i; f_c0 = 0).  With R(B) = L L^T (Cholesky,
// once) and G_i = L^{-1} D_i, the band's eigenvalues are those of the Hermitian
// C_i = G_i R(A0) G_i^*.  Per group of bands: G_i by a kernel, two batched
// complex GEMMs, then one Hermitian eigenvalue solve per band (cuSOLVER,
// eigenvalues only).  O(I N^3): meant for small N (the paper's adaptive
// baseline solves exactly these GEPs), as a check of the L-hat / E-hat
// estimates.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace m2 {
namespace {

constexpr double kPiT = 3.141592653589793238462643383279502884;

// column-major N x N real: RB (signal band |f| <= fmax) and RA (|f| <= f_w)
__global__ void ts_matrices_kernel(const double* __restrict__ t, int N, double fmax, double fw,
                                   double* __restrict__ RB, double2* __restrict__ RA) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= N) return;
    const size_t o = (size_t)i + (size_t)j * N;
    if (i == j) {
        RB[o] = 2.0 * fmax;
        RA[o] = make_double2(2.0 * fw, 0.0);
        return;
    }
    const double d = t[i] - t[j];
    RB[o] = sinpi(2.0 * fmax * d) / (kPiT * d);
    RA[o] = make_double2(sinpi(2.0 * fw * d) / (kPiT * d), 0.0);
}

// G_b[r][c] = Linv[r][c] e^{i 2 pi f_b t_c} for the bands of the group (column-major)
__global__ void g_kernel(int N, const double* __restrict__ Linv, const double* __restrict__ t,
                         const double* __restrict__ f, double2* __restrict__ G) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    const int b = blockIdx.z;
    if (r >= N) return;
    double s, co;
    sincospi(2.0 * f[b] * t[c], &s, &co);
    const double l = Linv[(size_t)c * N + r];
    G[(size_t)b * N * N + (size_t)c * N + r] = make_double2(l * co, l * s);
}

}  // namespace
}  // namespace m2

extern "C" m2_status m2nufft_true_suboptimality(m2nufft_plan_t p, double* E, double* lam_band) {
    using namespace m2;
    clear_error();
    if (!p || !E) {
        set_error("m2nufft_true_suboptimality: plan or E is NULL");
        return M2_ERR_ARG;
    }
    if (!p->have_lambda || p->complex_taper) {
        set_error("m2nufft_true_suboptimality: needs a full-band plan with nominal eigenvalues");
        return M2_ERR_ARG;
    }
    const int64_t N64 = p->g.N, I = p->g.I;
    const int K = p->g.K;
    if (N64 > 512 || (double)I * (double)N64 * N64 * N64 > 4e12) {
        set_error("m2nufft_true_suboptimality: O(I N^3) per-band GEPs are limited to N <= 512 and I N^3 <= 4e12");
        return M2_ERR_ARG;
    }
    const int N = (int)N64;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != p->device) M2_CUDA_TRY(cudaSetDevice(p->device));
    struct Restore {
        int dev, prev;
        ~Restore() {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{p->device, prev};

    // centred times: the eigenvalues do not depend on the time origin
    std::vector<double> tc(p->t);
    double tbar = 0;
    for (double v : tc) tbar += v;
    tbar /= (double)N;
    for (double& v : tc) v -= tbar;
    const int group = (int)std::max<int64_t>(1, std::min<int64_t>(I, (int64_t(256) << 20) / ((int64_t)N * N * 16 * 3)));

    std::vector<void*> owned;
    struct Free {
        std::vector<void*>* o;
        ~Free() {
            for (void* q : *o) cudaFree(q);
        }
    } freer{&owned};
    auto alloc = [&](void** ptr, size_t bytes) {
        cudaError_t e = cudaMalloc(ptr, std::max<size_t>(bytes, 8));
        if (e == cudaSuccess) owned.push_back(*ptr);
        return e;
    };
    double *dt = nullptr, *RB = nullptr, *Linv = nullptr, *dW = nullptr, *df = nullptr, *wk = nullptr;
    double2 *RA = nullptr, *G = nullptr, *T = nullptr, *C = nullptr, *zwork = nullptr;
    int* dinfo = nullptr;
    M2_CUDA_TRY(alloc((void**)&dt, sizeof(double) * N));
    M2_CUDA_TRY(alloc((void**)&RB, sizeof(double) * N * N));
    M2_CUDA_TRY(alloc((void**)&Linv, sizeof(double) * N * N));
    M2_CUDA_TRY(alloc((void**)&RA, sizeof(double2) * N * N));
    M2_CUDA_TRY(alloc((void**)&G, sizeof(double2) * (size_t)group * N * N));
    M2_CUDA_TRY(alloc((void**)&T, sizeof(double2) * (size_t)group * N * N));
    M2_CUDA_TRY(alloc((void**)&C, sizeof(double2) * (size_t)group * N * N));
    M2_CUDA_TRY(alloc((void**)&dW, sizeof(double) * (size_t)group * N));
    M2_CUDA_TRY(alloc((void**)&df, sizeof(double) * group));
    M2_CUDA_TRY(alloc((void**)&dinfo, sizeof(int) * (size_t)group));
    M2_CUDA_TRY(cudaMemcpy(dt, tc.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    ts_matrices_kernel<<<dim3((N + 127) / 128, N), 128>>>(dt, N, 0.5 * p->fs, p->f_w, RB, RA);
    M2_CUDA_TRY(cudaGetLastError());

    cusolverDnHandle_t hs = nullptr;
    cublasHandle_t hb = nullptr;
    struct Handles {
        cusolverDnHandle_t* s;
        cublasHandle_t* b;
        ~Handles() {
            if (*s) cusolverDnDestroy(*s);
            if (*b) cublasDestroy(*b);
        }
    } handles{&hs, &hb};
    if (cusolverDnCreate(&hs) != CUSOLVER_STATUS_SUCCESS || cublasCreate(&hb) != CUBLAS_STATUS_SUCCESS) {
        set_error("m2nufft_true_suboptimality: cuSOLVER/cuBLAS handle creation failed");
        return M2_ERR_CUDA;
    }
    // R(B) = L L^T, Linv = L^{-1}
    int lw = 0, info = 0;
    if (cusolverDnDpotrf_bufferSize(hs, CUBLAS_FILL_MODE_LOWER, N, RB, N, &lw) != CUSOLVER_STATUS_SUCCESS) {
        set_error("m2nufft_true_suboptimality: potrf buffer size failed");
        return M2_ERR_GEP;
    }
    M2_CUDA_TRY(alloc((void**)&wk, sizeof(double) * std::max(lw, 1)));
    if (cusolverDnDpotrf(hs, CUBLAS_FILL_MODE_LOWER, N, RB, N, wk, lw, dinfo) != CUSOLVER_STATUS_SUCCESS) {
        set_error("m2nufft_true_suboptimality: Cholesky of R(B) failed");
        return M2_ERR_GEP;
    }
    M2_CUDA_TRY(cudaMemcpy(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost));
    if (info != 0) {
        set_error("m2nufft_true_suboptimality: R(B) is not positive definite in FP64 (info %d)", info);
        return M2_ERR_GEP;
    }
    {
        std::vector<double> eye((size_t)N * N, 0.0);
        for (int i = 0; i < N; ++i) eye[(size_t)i * N + i] = 1.0;
        M2_CUDA_TRY(cudaMemcpy(Linv, eye.data(), sizeof(double) * N * N, cudaMemcpyHostToDevice));
        const double one = 1.0;
        if (cublasDtrsm(hb, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, N, N, &one,
                        RB, N, Linv, N) != CUBLAS_STATUS_SUCCESS) {
            set_error("m2nufft_true_suboptimality: triangular inverse failed");
            return M2_ERR_CUDA;
        }
    }
    int lwz = 0;
    if (cusolverDnZheevd_bufferSize(hs, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, N,
                                    reinterpret_cast<cuDoubleComplex*>(C), N, dW, &lwz) != CUSOLVER_STATUS_SUCCESS) {
        set_error("m2nufft_true_suboptimality: heevd buffer size failed");
        return M2_ERR_GEP;
    }
    M2_CUDA_TRY(alloc((void**)&zwork, sizeof(double2) * std::max(lwz, 1)));
    std::vector<double> w((size_t)group * N), lb((size_t)I * K);
    std::vector<int> infos(group);
    const cuDoubleComplex one = {1.0, 0.0}, zero = {0.0, 0.0};
    for (int64_t i0 = 0; i0 < I; i0 += group) {
        const int nb = (int)std::min<int64_t>(group, I - i0);
        std::vector<double> f(nb);
        for (int b = 0; b < nb; ++b) f[b] = p->g.f_lo + (double)(i0 + b) * p->g.df;
        M2_CUDA_TRY(cudaMemcpy(df, f.data(), sizeof(double) * nb, cudaMemcpyHostToDevice));
        g_kernel<<<dim3((N + 127) / 128, N, nb), 128>>>(N, Linv, dt, df, G);
        M2_CUDA_TRY(cudaGetLastError());
        const long long st = (long long)N * N;
        if (cublasZgemmStridedBatched(hb, CUBLAS_OP_N, CUBLAS_OP_N, N, N, N, &one,
                                      reinterpret_cast<cuDoubleComplex*>(G), N, st,
                                      reinterpret_cast<cuDoubleComplex*>(RA), N, 0, &zero,
                                      reinterpret_cast<cuDoubleComplex*>(T), N, st, nb) != CUBLAS_STATUS_SUCCESS ||
            cublasZgemmStridedBatched(hb, CUBLAS_OP_N, CUBLAS_OP_C, N, N, N, &one,
                                      reinterpret_cast<cuDoubleComplex*>(T), N, st,
                                      reinterpret_cast<cuDoubleComplex*>(G), N, st, &zero,
                                      reinterpret_cast<cuDoubleComplex*>(C), N, st, nb) != CUBLAS_STATUS_SUCCESS) {
            set_error("m2nufft_true_suboptimality: batched GEMM failed");
            return M2_ERR_CUDA;
        }
        // one eigenvalue solve per band, results gathered once per group
        for (int b = 0; b < nb; ++b) {
            if (cusolverDnZheevd(hs, CUSOLVER_EIG_MODE_NOVECTOR, CUBLAS_FILL_MODE_LOWER, N,
                                 reinterpret_cast<cuDoubleComplex*>(C) + (size_t)b * N * N, N, dW + (size_t)b * N,
                                 reinterpret_cast<cuDoubleComplex*>(zwork), lwz, dinfo + b) != CUSOLVER_STATUS_SUCCESS) {
                set_error("m2nufft_true_suboptimality: heevd failed");
                return M2_ERR_GEP;
            }
        }
        M2_CUDA_TRY(cudaMemcpy(w.data(), dW, sizeof(double) * (size_t)nb * N, cudaMemcpyDeviceToHost));
        M2_CUDA_TRY(cudaMemcpy(infos.data(), dinfo, sizeof(int) * nb, cudaMemcpyDeviceToHost));
        for (int b = 0; b < nb; ++b) {
            if (infos[b] != 0) {
                set_error("m2nufft_true_suboptimality: band %lld eigenvalues did not converge (info %d)",
                          (long long)(i0 + b), infos[b]);
                return M2_ERR_GEP;
            }
            for (int k = 0; k < K; ++k) lb[(size_t)(i0 + b) * K + k] = w[(size_t)b * N + N - 1 - k];
        }
    }
    for (int64_t i = 0; i < I; ++i) {
        double s = 0;
        for (int k = 0; k < K; ++k) s += std::fabs(lb[(size_t)i * K + k] - p->lambda[k]);
        E[i] = s / K;
    }
    if (lam_band) std::memcpy(lam_band, lb.data(), sizeof(double) * lb.size());
    return M2_OK;
}
