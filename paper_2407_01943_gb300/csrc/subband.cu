// Nominal tapers of one sub-band (Sec. 2.3 and the multiband partition of
// Sec. 3): the GEP R(A0) w = lambda R(B^q) w (Eq. gep_at_A0) with the nominal
// band A0 = {|f - f_c0| <= f_w} inside the sub-band B^q = {f_min <= |f| <= f_max}.
//
//   R(B^q | n, m) = 2 cos(pi (f_max + f_min) d) sin(pi (f_max - f_min) d) / (pi d)   (Eq. gpss_matrix_b_q)
//   R(A0 | n, m)  = sin(2 pi f_w d) / (pi d) e^{i 2 pi f_c0 d}                      (Eq. gpss_matrix_a)
//
// R(B^q) is positive definite in exact arithmetic but numerically singular
// once N exceeds the sub-band's Shannon number 2 (f_max - f_min) T, so the GEP
// is solved on its numerical range: R(B^q) = U S U^T (FP64 cuSOLVER), keep the
// eigenvalues above kRangeTol times the largest (r of them), M = U_r S_r^{-1/2},
// C = M^T R(A0) M (Hermitian r x r; cuBLAS, real and imaginary parts apart),
// the K largest eigenpairs C y = lambda y (cuSOLVER), w = M y sqrt(2 f_w), so
// that w^H R(B^q) w = 2 f_w (Eq. bg_norm_requirement).  Since A0 lies inside
// B^q, R(B^q) - R(A0) is positive semi-definite and the discarded directions
// carry no energy in A0 either.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace m2 {
namespace {

constexpr double kPiS = 3.141592653589793238462643383279502884;
constexpr double kRangeTol = 1e-9;

// column-major N x N: RB (real), RA split into real and imaginary parts
__global__ void subband_matrices_kernel(const double* __restrict__ t, int N, double f_w, double f_c0, double f_min,
                                        double f_max, double* __restrict__ RB, double* __restrict__ RAr,
                                        double* __restrict__ RAi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= N) return;
    const size_t o = (size_t)i + (size_t)j * N;
    if (i == j) {
        RB[o] = 2.0 * (f_max - f_min);
        RAr[o] = 2.0 * f_w;
        RAi[o] = 0.0;
        return;
    }
    const double d = t[i] - t[j];
    const double pd = kPiS * d;
    RB[o] = 2.0 * cospi((f_max + f_min) * d) * sinpi((f_max - f_min) * d) / pd;
    const double a = sinpi(2.0 * f_w * d) / pd;
    double sn, cs;
    sincospi(2.0 * f_c0 * d, &sn, &cs);
    RAr[o] = a * cs;
    RAi[o] = a * sn;
}

// M[:, c] = U[:, off + c] / sqrt(s[off + c])
__global__ void scale_columns_kernel(int N, int r, int off, const double* __restrict__ U,
                                     const double* __restrict__ s, double* __restrict__ M) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= N) return;
    M[(size_t)c * N + i] = U[(size_t)(off + c) * N + i] * rsqrt(s[off + c]);
}

// C = (Cr + Cr^T)/2 + i (Ci - Ci^T)/2 as cuDoubleComplex (Hermitian part of Cr + i Ci)
__global__ void hermitian_kernel(int r, const double* __restrict__ Cr, const double* __restrict__ Ci,
                                 double2* __restrict__ C) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= r) return;
    const size_t o = (size_t)i + (size_t)j * r, ot = (size_t)j + (size_t)i * r;
    C[o] = make_double2(0.5 * (Cr[o] + Cr[ot]), 0.5 * (Ci[o] - Ci[ot]));
}

// split complex Y (r x K) into real parts
__global__ void split_kernel(int n, const double2* __restrict__ Y, double* __restrict__ Yr, double* __restrict__ Yi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Yr[i] = Y[i].x;
    Yi[i] = Y[i].y;
}

struct Scratch {
    std::vector<void*> p;
    ~Scratch() {
        for (void* q : p) cudaFree(q);
    }
    template <typename T>
    cudaError_t alloc(T** out, size_t n) {
        cudaError_t e = cudaMalloc(out, sizeof(T) * std::max<size_t>(n, 1));
        if (e == cudaSuccess) p.push_back(*out);
        return e;
    }
};

}  // namespace

m2_status solve_gep_subband(const std::vector<double>& ts, double f_w, int K, double f_c0, double f_min,
                            double f_max, size_t budget, std::vector<double>& w_re, std::vector<double>& w_im,
                            std::vector<double>& lam, double& seconds) {
    const auto t0 = std::chrono::steady_clock::now();
    const int N = (int)ts.size();
    const size_t mat = (size_t)N * N;
    if (budget && 5 * mat * sizeof(double) > budget) {
        set_error("sub-band GEP needs %zu bytes, above mem_budget", 5 * mat * sizeof(double));
        return M2_ERR_BUDGET;
    }
    Scratch sc;
    double *dt, *RB, *RAr, *RAi, *s;
    int* dinfo;
#define SB_CUDA(expr)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            set_error("sub-band GEP: %s failed: %s", #expr, cudaGetErrorString(e_));       \
            return e_ == cudaErrorMemoryAllocation ? M2_ERR_NOMEM : M2_ERR_CUDA;           \
        }                                                                                  \
    } while (0)
    SB_CUDA(sc.alloc(&dt, N));
    SB_CUDA(sc.alloc(&RB, mat));
    SB_CUDA(sc.alloc(&RAr, mat));
    SB_CUDA(sc.alloc(&RAi, mat));
    SB_CUDA(sc.alloc(&s, N));
    SB_CUDA(sc.alloc(&dinfo, 1));
    SB_CUDA(cudaMemcpy(dt, ts.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    subband_matrices_kernel<<<dim3((N + 255) / 256, N), 256>>>(dt, N, f_w, f_c0, f_min, f_max, RB, RAr, RAi);
    SB_CUDA(cudaGetLastError());

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
        set_error("sub-band GEP: cuSOLVER/cuBLAS handle creation failed");
        return M2_ERR_CUDA;
    }
    // R(B^q) = U S U^T (ascending eigenvalues, U overwrites RB)
    int lwork = 0, info = 0;
    if (cusolverDnDsyevd_bufferSize(hs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, N, RB, N, s, &lwork) !=
        CUSOLVER_STATUS_SUCCESS) {
        set_error("sub-band GEP: cusolverDnDsyevd_bufferSize failed");
        return M2_ERR_GEP;
    }
    double* work;
    SB_CUDA(sc.alloc(&work, (size_t)lwork));
    if (cusolverDnDsyevd(hs, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, N, RB, N, s, work, lwork, dinfo) !=
        CUSOLVER_STATUS_SUCCESS) {
        set_error("sub-band GEP: cusolverDnDsyevd failed");
        return M2_ERR_GEP;
    }
    SB_CUDA(cudaMemcpy(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost));
    if (info != 0) {
        set_error("sub-band GEP: eigendecomposition of R(B^q) did not converge (info %d)", info);
        return M2_ERR_GEP;
    }
    std::vector<double> hs_s(N);
    SB_CUDA(cudaMemcpy(hs_s.data(), s, sizeof(double) * N, cudaMemcpyDeviceToHost));
    const double smax = hs_s[N - 1];
    int off = 0;
    while (off < N && !(hs_s[off] > kRangeTol * smax)) ++off;
    const int r = N - off;
    if (r < K) {
        set_error("sub-band GEP: K = %d exceeds the numerical rank %d of R(B^q)", K, r);
        return M2_ERR_GEP;
    }
    double *M, *T, *Cr, *Ci;
    SB_CUDA(sc.alloc(&M, (size_t)N * r));
    SB_CUDA(sc.alloc(&T, (size_t)N * r));
    SB_CUDA(sc.alloc(&Cr, (size_t)r * r));
    SB_CUDA(sc.alloc(&Ci, (size_t)r * r));
    scale_columns_kernel<<<dim3((N + 255) / 256, r), 256>>>(N, r, off, RB, s, M);
    SB_CUDA(cudaGetLastError());
    const double one = 1.0, zero = 0.0;
    // C_r = M^T RAr M, C_i = M^T RAi M
    for (int part = 0; part < 2; ++part) {
        const double* A = part ? RAi : RAr;
        double* C = part ? Ci : Cr;
        if (cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, N, r, N, &one, A, N, M, N, &zero, T, N) != CUBLAS_STATUS_SUCCESS ||
            cublasDgemm(hb, CUBLAS_OP_T, CUBLAS_OP_N, r, r, N, &one, M, N, T, N, &zero, C, r) != CUBLAS_STATUS_SUCCESS) {
            set_error("sub-band GEP: cublasDgemm failed");
            return M2_ERR_CUDA;
        }
    }
    double2* C;
    double* w;
    SB_CUDA(sc.alloc(&C, (size_t)r * r));
    SB_CUDA(sc.alloc(&w, (size_t)r));
    hermitian_kernel<<<dim3((r + 255) / 256, r), 256>>>(r, Cr, Ci, C);
    SB_CUDA(cudaGetLastError());
    int meig = 0, lw2 = 0;
    if (cusolverDnZheevdx_bufferSize(hs, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER, r,
                                     reinterpret_cast<cuDoubleComplex*>(C), r, 0.0, 0.0, r - K + 1, r, &meig, w,
                                     &lw2) != CUSOLVER_STATUS_SUCCESS) {
        set_error("sub-band GEP: cusolverDnZheevdx_bufferSize failed");
        return M2_ERR_GEP;
    }
    double2* work2;
    SB_CUDA(sc.alloc(&work2, (size_t)lw2));
    if (cusolverDnZheevdx(hs, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_LOWER, r,
                          reinterpret_cast<cuDoubleComplex*>(C), r, 0.0, 0.0, r - K + 1, r, &meig, w,
                          reinterpret_cast<cuDoubleComplex*>(work2), lw2, dinfo) != CUSOLVER_STATUS_SUCCESS) {
        set_error("sub-band GEP: cusolverDnZheevdx failed");
        return M2_ERR_GEP;
    }
    SB_CUDA(cudaMemcpy(&info, dinfo, sizeof(int), cudaMemcpyDeviceToHost));
    if (info != 0 || meig != K) {
        set_error("sub-band GEP: reduced eigenproblem failed (info %d, %d of %d pairs)", info, meig, K);
        return M2_ERR_GEP;
    }
    // w = M y: the first K columns of C hold y (ascending eigenvalues)
    double *Yr, *Yi, *Wr, *Wi;
    SB_CUDA(sc.alloc(&Yr, (size_t)r * K));
    SB_CUDA(sc.alloc(&Yi, (size_t)r * K));
    SB_CUDA(sc.alloc(&Wr, (size_t)N * K));
    SB_CUDA(sc.alloc(&Wi, (size_t)N * K));
    split_kernel<<<(r * K + 255) / 256, 256>>>(r * K, C, Yr, Yi);
    SB_CUDA(cudaGetLastError());
    if (cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, N, K, r, &one, M, N, Yr, r, &zero, Wr, N) != CUBLAS_STATUS_SUCCESS ||
        cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_N, N, K, r, &one, M, N, Yi, r, &zero, Wi, N) != CUBLAS_STATUS_SUCCESS) {
        set_error("sub-band GEP: cublasDgemm (back-transform) failed");
        return M2_ERR_CUDA;
    }
    std::vector<double> hr((size_t)N * K), hi((size_t)N * K), hw(K);
    SB_CUDA(cudaMemcpy(hr.data(), Wr, sizeof(double) * hr.size(), cudaMemcpyDeviceToHost));
    SB_CUDA(cudaMemcpy(hi.data(), Wi, sizeof(double) * hi.size(), cudaMemcpyDeviceToHost));
    SB_CUDA(cudaMemcpy(hw.data(), w, sizeof(double) * K, cudaMemcpyDeviceToHost));
#undef SB_CUDA
    const double scl = std::sqrt(2.0 * f_w);
    w_re.assign((size_t)K * N, 0.0);
    w_im.assign((size_t)K * N, 0.0);
    lam.assign(K, 0.0);
    for (int k = 0; k < K; ++k) {
        const int src = K - 1 - k;  // descending
        lam[k] = hw[src];
        for (int n = 0; n < N; ++n) {
            w_re[(size_t)k * N + n] = hr[(size_t)src * N + n] * scl;
            w_im[(size_t)k * N + n] = hi[(size_t)src * N + n] * scl;
        }
    }
    seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return M2_OK;
}

}  // namespace m2
