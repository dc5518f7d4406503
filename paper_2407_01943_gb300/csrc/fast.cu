// Packed FP32 exec path (real tapers, nf = n1 * 1024, support <= 64 rows).
//
// Same mathematics as the generic path in exec.cu (Sec. 3.2, Eq.
// eigencoefficients and Eq. power_spectrum_estimator evaluated by a type-1
// nonuniform FFT), organised for throughput:
//
//   * two real tapers share one complex FFT: the spread grid of taper pair j
//     is g_{2j} + i g_{2j+1}; since both grids are real, their transforms are
//     recovered from the packed transform Zp at k and nf - k:
//         X_{2j}[k]   = (Zp[k] + conj(Zp[nf-k])) / 2
//         X_{2j+1}[k] = (Zp[k] - conj(Zp[nf-k])) / (2i)
//     which halves the FFT work and the L2-resident workspace;
//   * the column DFTs (length n1, only `rows` nonzero inputs) are evaluated per
//     coset k1 = r + C q (C = n1/F, F = min(n1, 32)): the inputs are folded
//     modulo F with the twiddle W_n1^{l1 r} and one F-point FFT runs in
//     registers, one column per lane, so loads and stores are 256-byte rows;
//   * the 1024-point row DFTs run one per warp as 32 x 32 in registers with a
//     single padded shared-memory transpose;
//   * the epilogue pairs each row k1 with its mirror n1 - k1 inside the CTA,
//     unpacks, deconvolves, writes J and |J|^2 with streaming stores, and sums
//     P-hat over all taper pairs in registers (no atomics).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace m2 {
namespace {

constexpr int kRowLen = 1024;     // n2 of the packed path
constexpr int kRowPad = 1060;     // per-warp transpose / row buffer: >= 32 x 33, and 2*1060 = 8 (mod 32)
                                  // words so the epilogue's 4 rows x 4 columns per half-warp hit
                                  // 32 distinct banks
constexpr int kColWarps = 4;      // warps per CTA of the column pass

struct Tw32 {
    float2 w[16];  // exp(-i 2 pi e / 32), e < 16
};

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__host__ __device__ constexpr int brev(int v, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((v >> i) & 1) << (bits - 1 - i);
    return r;
}
__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// In-register radix-2 decimation-in-frequency FFT of length N <= 32 (natural
// input, bit-reversed output): v[q] holds X[brev(q)].
template <int N>
__device__ __forceinline__ void fft_reg(float2 (&v)[N], const Tw32& tw) {
#pragma unroll
    for (int h = N / 2; h >= 1; h /= 2) {
#pragma unroll
        for (int blk = 0; blk < N; blk += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const float2 a = v[blk + j], b = v[blk + j + h];
                v[blk + j] = make_float2(a.x + b.x, a.y + b.y);
                const float2 d = make_float2(a.x - b.x, a.y - b.y);
                const int e = j * (32 / (2 * h));
                if (e == 0) v[blk + j + h] = d;
                else if (e == 8) v[blk + j + h] = make_float2(d.y, -d.x);
                else v[blk + j + h] = cmulf(d, tw.w[e]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// spread (packed): gp[b][j][c] = sum_n (u_{2j}[n] + i u_{2j+1}[n]) x_b[n] phi(c - u_n)
// ---------------------------------------------------------------------------
template <int KP>
__global__ void __launch_bounds__(kSpreadTile)
spread_packed_kernel(const float* __restrict__ x, int64_t N, const int32_t* __restrict__ pt_src,
                     const int32_t* __restrict__ pt_cell, const float* __restrict__ pt_off,
                     const float* __restrict__ taper, int64_t P, const int32_t* __restrict__ tile_pb,
                     const int32_t* __restrict__ tile_pe, int K, int Kp, int w, float two_over_w, float beta,
                     int64_t Lg, float2* __restrict__ g) {
    __shared__ int32_t s_cell[kSpreadChunk];
    __shared__ float s_off[kSpreadChunk];
    __shared__ float2 s_val[KP][kSpreadChunk];
    const int tile = blockIdx.x;
    const int b = blockIdx.y;
    const int64_t c = (int64_t)tile * kSpreadTile + threadIdx.x;
    const int pb = tile_pb[tile], pe = tile_pe[tile];
    const float* xb = x + (int64_t)b * N;
    float2 acc[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) acc[j] = make_float2(0.f, 0.f);
    for (int q0 = pb; q0 < pe; q0 += kSpreadChunk) {
        const int n = min(kSpreadChunk, pe - q0);
        __syncthreads();
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int p = q0 + t;
            s_cell[t] = pt_cell[p];
            s_off[t] = pt_off[p];
            const float xv = xb[pt_src[p]];
#pragma unroll
            for (int j = 0; j < KP; ++j) {
                float2 v = make_float2(0.f, 0.f);
                if (2 * j < K) v.x = taper[(int64_t)(2 * j) * P + p] * xv;
                if (2 * j + 1 < K) v.y = taper[(int64_t)(2 * j + 1) * P + p] * xv;
                s_val[j][t] = v;
            }
        }
        __syncthreads();
        if (c < Lg) {
            const int ci = (int)c;
            int lo = 0, hi = n;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_cell[mid] + w <= ci) lo = mid + 1; else hi = mid;
            }
            for (int t = lo; t < n && s_cell[t] <= ci; ++t) {
                const float z = s_off[t] + (float)(ci - s_cell[t]);
                const float a = z * two_over_w;
                const float phi = expf(beta * (sqrtf(fmaxf(0.f, 1.f - a * a)) - 1.f));
#pragma unroll
                for (int j = 0; j < KP; ++j) {
                    acc[j].x += s_val[j][t].x * phi;
                    acc[j].y += s_val[j][t].y * phi;
                }
            }
        }
    }
    if (c < Lg) {
#pragma unroll
        for (int j = 0; j < KP; ++j)
            if (j < Kp) g[((int64_t)b * Kp + j) * Lg + c] = acc[j];
    }
}

// ---------------------------------------------------------------------------
// column pass: Z[b][j][k1][l2] = W_nf^{l2 k1} sum_{l1 < rows} gp[b][j][l1 n2 + l2] W_n1^{l1 k1}
// CTA = 32 columns x all cosets; lane = column; F-point FFT per coset in registers.
// The output twiddle W_nf^{l2 (r + C q)} = W_nf^{l2 r} * T_lane[q] uses a per-lane
// table T_lane[q] = W_nf^{l2 C q} stored [q][lane] (conflict-free) and one base
// factor per coset.
// ---------------------------------------------------------------------------
template <int F>
__global__ void __launch_bounds__(32 * kColWarps)
cols_fast_kernel(const float2* __restrict__ gp, int64_t Lg, int rows, int n1, int Kp,
                 const float2* __restrict__ tw_n1 /*[n1] full circle*/,
                 const float2* __restrict__ colT /*[F][1024]: W_nf^{l2 C q}*/,
                 const float2* __restrict__ colB /*[C][1024]: W_nf^{l2 r}*/, Tw32 tw, float2* __restrict__ Z) {
    extern __shared__ float2 smem_f2[];
    float2* s_in = smem_f2;           // [rows][32]
    float2* s_tw = s_in + rows * 32;  // [n1]
    float2* s_T = s_tw + n1;          // [F][32]
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int l2 = blockIdx.x * 32 + lane;
    const int j = blockIdx.y;
    const int b = blockIdx.z;
    const int64_t n2 = kRowLen;
    const int C = n1 / F;
    const float2* gj = gp + ((int64_t)b * Kp + j) * Lg;
    float2* Zj = Z + ((int64_t)b * Kp + j) * (int64_t)n1 * n2;

    for (int l1 = warp; l1 < rows; l1 += kColWarps) s_in[l1 * 32 + lane] = gj[(int64_t)l1 * n2 + l2];
    for (int q = threadIdx.x; q < n1; q += blockDim.x) s_tw[q] = tw_n1[q];
    for (int q = warp; q < F; q += kColWarps) s_T[q * 32 + lane] = colT[q * kRowLen + l2];
    __syncthreads();

    const int nfold = (rows + F - 1) / F;
    for (int r = warp; r < C; r += kColWarps) {
        const float2 base = colB[(int64_t)r * kRowLen + l2];
        float2 v[F];
#pragma unroll
        for (int q = 0; q < F; ++q) v[q] = make_float2(0.f, 0.f);
        int tix = 0;  // (l1 * r) mod n1, advanced incrementally
        for (int f = 0; f < nfold; ++f) {
#pragma unroll
            for (int q = 0; q < F; ++q) {
                const int l1 = f * F + q;
                if (l1 < rows) {
                    const float2 a = s_in[l1 * 32 + lane];
                    const float2 t = s_tw[tix];
                    v[q].x += a.x * t.x - a.y * t.y;
                    v[q].y += a.x * t.y + a.y * t.x;
                }
                tix += r;
                if (tix >= n1) tix -= n1;
            }
        }
        fft_reg<F>(v, tw);
#pragma unroll
        for (int q = 0; q < F; ++q) {
            const int k1 = r + C * q;
            const float2 t = cmulf(base, s_T[q * 32 + lane]);
            Zj[(int64_t)k1 * n2 + l2] = cmulf(v[brev(q, ilog2c(F))], t);
        }
    }
}

// ---------------------------------------------------------------------------
// row pass: X[k1 + n1 k2] = sum_{l2} Z[k1][l2] W_1024^{l2 k2}, written transposed as
// Xt[k2][k1] so that the epilogue reads and writes long contiguous runs.
// CTA = R consecutive rows of one (signal, pair); one warp per row, 32 x 32 in
// registers with one padded shared-memory transpose; the transformed rows are
// staged in shared memory and written R rows at a time per k2.
// ---------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(32 * R, (R <= 8 ? 2 : 1))
rowfft_kernel(const float2* __restrict__ Z, int n1, int Kp, const float2* __restrict__ tw1024, Tw32 tw,
              int k2max, float2* __restrict__ Xt) {
    constexpr int NT = 32 * R;
    extern __shared__ float2 smem_f2[];
    float2* s_tw = smem_f2;          // [32 c][32 lane]: W_1024^{lane c}
    float2* s_row = s_tw + kRowLen;  // [R][kRowPad]
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int r0 = blockIdx.x * R;
    const int j = blockIdx.y;
    const int b = blockIdx.z;
    const int64_t base = ((int64_t)b * Kp + j) * (int64_t)n1 * kRowLen;

    for (int q = threadIdx.x; q < kRowLen; q += NT) s_tw[q] = tw1024[(q >> 5) * (q & 31)];

    const float2* Zr = Z + base + (int64_t)(r0 + warp) * kRowLen + lane;
    float2 v[32];
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = __ldcs(Zr + 32 * a);
    __syncthreads();  // s_tw ready
    float2* S = s_row + warp * kRowPad;
    fft_reg<32>(v, tw);  // over a for column b = lane: v[q] = Y[lane][brev(q)]
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const int c = brev(q, 5);
        S[c * 33 + lane] = cmulf(v[q], s_tw[c * 32 + lane]);
    }
    __syncwarp();
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = S[lane * 33 + a];
    __syncwarp();
    fft_reg<32>(v, tw);  // over b for column c = lane: v[q] = X[lane + 32 brev(q)]
#pragma unroll
    for (int q = 0; q < 32; ++q) S[lane + 32 * brev(q, 5)] = v[q];
    __syncthreads();
    // Xt[k2][r0 + rr] for rr < R: consecutive threads take consecutive rows.  Only the
    // columns the epilogue reads are written: k2 <= k2max and their partners k2 >= 1023 - k2max
    // (and 1024 - k2 for row 0, which lies in the same two ranges).
    float2* Xb = Xt + base + r0;
    const int nlo = k2max + 1;                  // k2 in [0, nlo)
    const int nout = 2 * nlo;                   // plus k2 in [1024 - nlo, 1024)
#pragma unroll 4
    for (int e = threadIdx.x; e < R * nout; e += NT) {
        const int rr = e % R, q = e / R;
        const int k2 = q < nlo ? q : kRowLen - nout + q;
        Xb[(int64_t)k2 * n1 + rr] = s_row[rr * kRowPad + k2];
    }
}

// ---------------------------------------------------------------------------
// epilogue: unpack the taper pairs, deconvolve, write J and |J|^2, average P-hat.
// Thread = position k = k1 + n1 k2 with k2 <= k2max (k in the upper half-spectrum
// side m >= 0) together with its partner nf - k = (n1 - k1, 1023 - k2), or
// (0, 1024 - k2) for k1 = 0.  Both tapers of a pair are real, so X(nf - k) =
// conj X(k) per taper and s(-m) = conj s(m): one thread computes J at k and
// writes J(m) and conj J(m) = J(-m).  The deconvolution factor is loaded once
// and reused for all K/2 pairs; P-hat is summed in registers.  Consecutive
// threads take consecutive k1, so every load and store is a contiguous run.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
epi_kernel(const float2* __restrict__ Xt, int n1, int Kp, int K, int I, int i_c, int nf,
           const float2* __restrict__ deconv, float2* __restrict__ J, float* __restrict__ E,
           float* __restrict__ Pout) {
    const int k1 = blockIdx.x * blockDim.x + threadIdx.x;
    const int k2 = blockIdx.y;
    const int b = blockIdx.z;
    if (k1 >= n1) return;
    const int half = nf >> 1;
    int pk1, pk2;
    if (k1 == 0) {
        pk1 = 0;
        pk2 = (kRowLen - k2) & (kRowLen - 1);
    } else {
        pk1 = n1 - k1;
        pk2 = kRowLen - 1 - k2;
    }
    const int kk1 = k1 + n1 * k2;
    const int kk2 = pk1 + n1 * pk2;
    const int i1 = (kk1 < half ? kk1 : kk1 - nf) + i_c;
    const int i2 = (kk2 < half ? kk2 : kk2 - nf) + i_c;
    const bool v1 = (unsigned)i1 < (unsigned)I;
    const bool v2 = (unsigned)i2 < (unsigned)I && kk2 != kk1;
    if (!v1 && !v2) return;
    float2 sd;
    if (v1) {
        sd = __ldg(deconv + i1);
    } else {
        sd = __ldg(deconv + i2);
        sd.y = -sd.y;
    }
    const int64_t plane = (int64_t)n1 * kRowLen;
    const float2* X1 = Xt + (int64_t)b * Kp * plane + (int64_t)k2 * n1 + k1;
    const float2* X2 = Xt + (int64_t)b * Kp * plane + (int64_t)pk2 * n1 + pk1;
    float pacc = 0.f;
    for (int j = 0; j < Kp; ++j) {
        const float2 A = __ldcs(X1 + (int64_t)j * plane);
        const float2 Bc = __ldcs(X2 + (int64_t)j * plane);
        // X_even = (A + conj(B)) / 2 ; X_odd = (A - conj(B)) / (2i)
        const float2 j0 = cmulf(make_float2(0.5f * (A.x + Bc.x), 0.5f * (A.y - Bc.y)), sd);
        const float p0 = j0.x * j0.x + j0.y * j0.y;
        const int64_t o0 = ((int64_t)b * K + 2 * j) * I;
        if (J) {
            if (v1) __stcs(J + o0 + i1, j0);
            if (v2) __stcs(J + o0 + i2, make_float2(j0.x, -j0.y));
        }
        if (E) {
            if (v1) __stcs(E + o0 + i1, p0);
            if (v2) __stcs(E + o0 + i2, p0);
        }
        pacc += p0;
        if (2 * j + 1 < K) {
            const float2 j1 = cmulf(make_float2(0.5f * (A.y + Bc.y), -0.5f * (A.x - Bc.x)), sd);
            const float p1 = j1.x * j1.x + j1.y * j1.y;
            const int64_t o1 = o0 + I;
            if (J) {
                if (v1) __stcs(J + o1 + i1, j1);
                if (v2) __stcs(J + o1 + i2, make_float2(j1.x, -j1.y));
            }
            if (E) {
                if (v1) __stcs(E + o1 + i1, p1);
                if (v2) __stcs(E + o1 + i2, p1);
            }
            pacc += p1;
        }
    }
    if (Pout) {
        const float pv = pacc * (1.0f / (float)K);
        float* Pb = Pout + (int64_t)b * I;
        if (v1) __stcs(Pb + i1, pv);
        if (v2) __stcs(Pb + i2, pv);
    }
}

Tw32 make_tw32() {
    Tw32 t;
    for (int e = 0; e < 16; ++e) {
        const double a = 2.0 * 3.141592653589793238462643383279502884 * e / 32.0;
        t.w[e] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
    return t;
}

template <int KP>
m2_status launch_spread_packed(m2nufft_plan_s* p, const float* x, int nb, cudaStream_t st) {
    const Geometry& g = p->g;
    dim3 grid((unsigned)g.ntiles, (unsigned)nb);
    spread_packed_kernel<KP><<<grid, kSpreadTile, 0, st>>>(
        x, g.N, p->d_pt_src, p->d_pt_cell, reinterpret_cast<const float*>(p->d_pt_off),
        reinterpret_cast<const float*>(p->d_taper), g.P, p->d_tile_pb, p->d_tile_pe, g.K, g.kp, g.width,
        (float)(2.0 / g.width), (float)g.beta, g.Lg, reinterpret_cast<float2*>(p->d_g));
    M2_CUDA_TRY(cudaGetLastError());
    return M2_OK;
}

template <int F>
m2_status launch_cols_fast(m2nufft_plan_s* p, int nb, cudaStream_t st, const Tw32& tw) {
    const Geometry& g = p->g;
    const size_t smem = sizeof(float2) * ((size_t)g.rows * 32 + g.n1 + (size_t)F * 32);
    auto kern = cols_fast_kernel<F>;
    dim3 grid((unsigned)(kRowLen / 32), (unsigned)g.kp, (unsigned)nb);
    kern<<<grid, 32 * kColWarps, smem, st>>>(reinterpret_cast<const float2*>(p->d_g), g.Lg, (int)g.rows,
                                              (int)g.n1, g.kp, reinterpret_cast<const float2*>(p->d_twn1),
                                              reinterpret_cast<const float2*>(p->d_colT),
                                              reinterpret_cast<const float2*>(p->d_colB), tw,
                                              reinterpret_cast<float2*>(p->d_Z));
    M2_CUDA_TRY(cudaGetLastError());
    return M2_OK;
}

template <int R>
m2_status launch_rowfft(m2nufft_plan_s* p, int nb, cudaStream_t st, const Tw32& tw, int k2max) {
    const Geometry& g = p->g;
    const size_t smem = sizeof(float2) * ((size_t)kRowLen + (size_t)R * kRowPad);
    auto kern = rowfft_kernel<R>;
    dim3 grid((unsigned)(g.n1 / R), (unsigned)g.kp, (unsigned)nb);
    kern<<<grid, 32 * R, smem, st>>>(reinterpret_cast<const float2*>(p->d_Z), (int)g.n1, g.kp,
                                     reinterpret_cast<const float2*>(p->d_tw1024), tw, k2max,
                                     reinterpret_cast<float2*>(p->d_X));
    M2_CUDA_TRY(cudaGetLastError());
    return M2_OK;
}

}  // namespace

m2_status init_fast_kernels(int smem_optin) {
    const void* funcs[] = {
        (const void*)cols_fast_kernel<2>,  (const void*)cols_fast_kernel<4>, (const void*)cols_fast_kernel<8>,
        (const void*)cols_fast_kernel<16>, (const void*)cols_fast_kernel<32>, (const void*)rowfft_kernel<2>,
        (const void*)rowfft_kernel<4>,     (const void*)rowfft_kernel<8>,
    };
    for (const void* f : funcs)
        M2_CUDA_TRY(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin));
    return M2_OK;
}

m2_status exec_fast_chunk(m2nufft_plan_s* p, const float* x, int nb, float2* J, float* E, float* P, cudaStream_t st) {
    const Geometry& g = p->g;
    static const Tw32 tw = make_tw32();

    mark(p, 0, 0, st);
    if (g.kp <= 2) M2_TRY(launch_spread_packed<2>(p, x, nb, st));
    else if (g.kp <= 4) M2_TRY(launch_spread_packed<4>(p, x, nb, st));
    else M2_TRY(launch_spread_packed<8>(p, x, nb, st));
    mark(p, 0, 1, st);

    mark(p, 1, 0, st);
    int64_t fdiv = 1;
    while (fdiv < 32 && g.n1 % (fdiv * 2) == 0) fdiv *= 2;
    switch (fdiv) {
        case 2: M2_TRY(launch_cols_fast<2>(p, nb, st, tw)); break;
        case 4: M2_TRY(launch_cols_fast<4>(p, nb, st, tw)); break;
        case 8: M2_TRY(launch_cols_fast<8>(p, nb, st, tw)); break;
        case 16: M2_TRY(launch_cols_fast<16>(p, nb, st, tw)); break;
        default: M2_TRY(launch_cols_fast<32>(p, nb, st, tw)); break;
    }
    mark(p, 1, 1, st);

    // positions k = k1 + n1 k2 on the m >= 0 side: k2 <= k2max where n1 k2 < I - i_c
    const int k2max = (int)std::min<int64_t>(kRowLen / 2 - 1, (g.I - g.i_c + g.n1 - 1) / g.n1);
    mark(p, 2, 0, st);
    {
        int R = 1;  // rows per CTA: largest power of two <= 8 dividing n1
        while (R < 8 && g.n1 % (R * 2) == 0) R *= 2;
        if (R == 8) M2_TRY(launch_rowfft<8>(p, nb, st, tw, k2max));
        else if (R == 4) M2_TRY(launch_rowfft<4>(p, nb, st, tw, k2max));
        else M2_TRY(launch_rowfft<2>(p, nb, st, tw, k2max));
    }
    mark(p, 2, 1, st);

    mark(p, 3, 0, st);
    {
        dim3 grid((unsigned)((g.n1 + 127) / 128), (unsigned)(k2max + 1), (unsigned)nb);
        epi_kernel<<<grid, 128, 0, st>>>(reinterpret_cast<const float2*>(p->d_X), (int)g.n1, g.kp, g.K, (int)g.I,
                                         (int)g.i_c, (int)g.nf, reinterpret_cast<const float2*>(p->d_deconv), J,
                                         E, P);
        M2_CUDA_TRY(cudaGetLastError());
    }
    mark(p, 3, 1, st);
    return M2_OK;
}

}  // namespace m2
