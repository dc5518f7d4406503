// Allocation-free leakage estimate: m2nufft_leakage_static.
//
// Same quantity as the plan's leakage estimate (App. B, Eq. lambda_hat_ki):
//   D_k^i = sum_{n,m} w_k(t_n) w_k(t_m) R(B|n,m) cos(2 pi f_i (t_n - t_m)),
//   L_k^i = |lambda_k - lambda_k 2 f_w / D_k^i|,   E_i = (1/K) sum_k L_k^i,
// but computed without a plan and without allocating: the double sum is split
// over blocks of n, each block's partial D goes to a file-scope device array,
// and a second kernel adds the partials in a fixed block order.
#include <mutex>

#include "common.cuh"

namespace {

// Scratch for the partial sums: nblk x K x I doubles at most.  Every GPU that
// loads this library holds these 32 MiB until the process exits.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;
constexpr int64_t kStaticScratchDoubles = (int64_t)(kStaticScratchBytes / sizeof(double));
static __device__ __align__(256) double m2_static_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
constexpr int kRowsPerBlock = 64;  // values of n per partial sum
std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

constexpr double kPiS = 3.141592653589793238462643383279502884;

// Device address of the scratch array on the current device.  Looked up again on every call made
// outside stream capture (cheap once the module is loaded, and right again after a
// cudaDeviceReset has given the device a new context); during a capture the address cached by
// the last call on this device outside capture is used.
m2_status scratch_address(int dev, cudaStream_t st, double** out) {
    if (dev < 0 || dev >= kMaxDevices) {
        m2::set_error("m2nufft_leakage_static: device ordinal %d out of range", dev);
        return M2_ERR_ARG;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    M2_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, m2_static_scratch);
        if (e != cudaSuccess || !ptr) {
            m2::set_error("cudaGetSymbolAddress(static scratch) failed: %s", cudaGetErrorString(e));
            return M2_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<double*>(ptr);
    } else if (!g_scratch_ptr[dev]) {
        m2::set_error("m2nufft_leakage_static: the first call on a device must come before any stream capture");
        return M2_ERR_ARG;
    }
    *out = g_scratch_ptr[dev];
    return M2_OK;
}

// partial[blk][k][i] = sum over n in block blk, m in [0, N), of w_k(t_n) w_k(t_m) R(n,m) cos(2 pi f_i (t_n - t_m))
__global__ void leakage_partial_kernel(int N, int K, int64_t I, const double* __restrict__ t,
                                       const double* __restrict__ w, double fmax, double f_lo, double df,
                                       double* __restrict__ partial) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int blk = blockIdx.y;
    if (i >= I) return;
    const double f = f_lo + (double)i * df;
    double D[m2::kMaxK];
    for (int k = 0; k < K; ++k) D[k] = 0.0;
    const int n0 = blk * kRowsPerBlock, n1 = min(N, n0 + kRowsPerBlock);
    for (int n = n0; n < n1; ++n) {
        for (int m = 0; m < N; ++m) {
            double r;
            if (m == n) {
                r = 2.0 * fmax;
            } else {
                const double d = t[n] - t[m];
                r = sinpi(2.0 * fmax * d) / (kPiS * d) * cospi(2.0 * f * d);
            }
            for (int k = 0; k < K; ++k) D[k] += w[(int64_t)k * N + n] * w[(int64_t)k * N + m] * r;
        }
    }
    for (int k = 0; k < K; ++k) partial[((int64_t)blk * K + k) * I + i] = D[k];
}

__global__ void leakage_reduce_kernel(int nblk, int K, int64_t I, const double* __restrict__ partial,
                                      const double* __restrict__ lam, double fw, double* __restrict__ L,
                                      double* __restrict__ Eh) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I) return;
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        double D = 0.0;
        for (int b = 0; b < nblk; ++b) D += partial[((int64_t)b * K + k) * I + i];
        const double lh = lam[k] * 2.0 * fw / D;
        const double l = fabs(lam[k] - lh);
        L[(int64_t)k * I + i] = l;
        s += l;
    }
    Eh[i] = s / K;
}

}  // namespace

extern "C" m2_status m2nufft_leakage_static(const double* t, int64_t N, double fs, double f_w, int K,
                                            const m2_fgrid* fc, const double* w, const double* lambda,
                                            double* Lhat, double* Ehat, void* stream) {
    m2::clear_error();
    if (!t || !w || !lambda || !Lhat || !Ehat || !fc) {
        m2::set_error("m2nufft_leakage_static: NULL pointer argument");
        return M2_ERR_ARG;
    }
    if (N < 1 || N > (int64_t(1) << 20) || K < 1 || K > m2::kMaxK || !(fs > 0) || !(f_w > 0) || !(f_w < 0.5 * fs) ||
        fc->I < 1 || !(fc->df > 0)) {
        m2::set_error("m2nufft_leakage_static: need 1 <= N <= 2^20, 1 <= K <= %d, fs > 0, 0 < f_w < fs/2, "
                      "I >= 1 and df > 0",
                      m2::kMaxK);
        return M2_ERR_ARG;
    }
    const int64_t I = fc->I;
    // one partial sum per block of kRowsPerBlock values of n, as many blocks as fit the scratch
    // (I is compared before K * I is formed, so no product can wrap)
    if (I > kStaticScratchDoubles / K) {
        m2::set_error("m2nufft_leakage_static: K = %d, I = %lld: K * I exceeds the static scratch of %lld doubles "
                      "(%zu MiB)",
                      K, (long long)I, (long long)kStaticScratchDoubles, kStaticScratchBytes >> 20);
        return M2_ERR_ARG;
    }
    const int64_t want = (N + kRowsPerBlock - 1) / kRowsPerBlock;
    if (want > kStaticScratchDoubles / ((int64_t)K * I)) {
        m2::set_error("m2nufft_leakage_static: N = %lld needs %lld partial sums of K * I doubles, above the "
                      "static scratch of %zu MiB",
                      (long long)N, (long long)want, kStaticScratchBytes >> 20);
        return M2_ERR_ARG;
    }
    int dev = 0;
    M2_CUDA_TRY(cudaGetDevice(&dev));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double* scratch = nullptr;
    m2_status s = scratch_address(dev, st, &scratch);
    if (s != M2_OK) return s;
    const int nblk = (int)want;
    dim3 g1((unsigned)((I + 127) / 128), (unsigned)nblk);
    leakage_partial_kernel<<<g1, 128, 0, st>>>((int)N, K, I, t, w, 0.5 * fs, fc->f_lo, fc->df, scratch);
    M2_CUDA_TRY(cudaGetLastError());
    leakage_reduce_kernel<<<(unsigned)((I + 127) / 128), 128, 0, st>>>(nblk, K, I, scratch, lambda, f_w, Lhat, Ehat);
    M2_CUDA_TRY(cudaGetLastError());
    return M2_OK;
}
