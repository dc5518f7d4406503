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
constexpr int kRowsR = 8;         // low rows per CTA of the row pass (plus as many mirror rows): runs of
                                  // 8 consecutive bands, i.e. whole 32-byte sectors for |J|^2 and P-hat
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
// row pass + unpack + epilogue
// ---------------------------------------------------------------------------
// CTA t owns R low rows k1 = t R + lr (lr < R) and their mirrors n1 - k1; the
// mirror of k1 = 0 is replaced by the other self-paired row n1/2.  Warp s
// transforms the row of slot s (slots [0, R) low, [R, 2R) mirror).
template <int R>
__device__ __forceinline__ int slot_row(int slot, int t, int n1) {
    if (slot < R) return t * R + slot;
    const int k1 = t * R + (slot - R);
    return k1 == 0 ? (n1 >> 1) : n1 - k1;
}

// Epilogue symmetry: the two tapers of a pair are real, so X(nf - k) = conj(X(k)) for
// each of them, and the deconvolution factors satisfy s(-m) = conj(s(m)) (phi-hat is
// real and even).  Hence J(-m) = conj(J(m)), |J(-m)|^2 = |J(m)|^2 and P(-m) = P(m):
// each thread unpacks one position k of a low row (from Zp[k] and Zp[nf - k], the
// latter in the mirror row) and writes both the output at k and the one at nf - k.
// Rows 0 and n1/2 pair with themselves; the thread that owns them (CTA 0, lr = 0)
// walks row 0 for k2 in [0, 512] and row n1/2 for k2 in [0, 512).
template <int R>
__global__ void __launch_bounds__(64 * R, (R <= 4 ? 2 : 1))
rows_fast_kernel(const float2* __restrict__ Z, int n1, int Kp, int K, int I, int i_c, int nf,
                 const float2* __restrict__ tw1024 /*[1024] full circle*/, Tw32 tw,
                 const float2* __restrict__ deconv, float2* __restrict__ J, float* __restrict__ E,
                 float* __restrict__ Pout) {
    constexpr int NT = 64 * R;           // threads
    constexpr int STEP = NT / R;         // k2 stride between a thread's positions (64)
    constexpr int NIT = kRowLen / STEP;  // positions per thread (16; 17 for the self-paired owner)
    extern __shared__ float2 smem_f2[];
    float2* s_tw = smem_f2;              // [32 c][32 lane]: W_1024^{lane c}
    float2* s_row = s_tw + kRowLen;      // [2R][kRowPad]
    float* s_pacc = reinterpret_cast<float*>(s_row + 2 * R * kRowPad);  // [NIT + 1][NT], thread-private
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int t = blockIdx.x;
    const int b = blockIdx.y;
    const int half = nf >> 1;

    for (int q = threadIdx.x; q < kRowLen; q += NT) s_tw[q] = tw1024[(q >> 5) * (q & 31)];

    const int lr = threadIdx.x % R;
    const int k2_0 = threadIdx.x / R;
    const int rowL = t * R + lr;
    const bool self = rowL == 0;         // owner of the self-paired rows 0 and n1/2
    const int rowM = self ? (n1 >> 1) : n1 - rowL;
    const int offL = lr * kRowPad, offM = (R + lr) * kRowPad;
    const int npos = self ? NIT + 1 : NIT;

    float* pacc = s_pacc + threadIdx.x;  // pacc[it * NT]
    for (int it = 0; it < npos; ++it) pacc[it * NT] = 0.f;

    const int my_row = slot_row<R>(warp, t, n1);
    float2* S = s_row + warp * kRowPad;
    const float2* Zrow = Z + ((int64_t)b * Kp * n1 + my_row) * kRowLen + lane;
    const int64_t zpair = (int64_t)n1 * kRowLen;  // stride between taper pairs

    // row of pair 0, prefetched into registers; the next pair's row is loaded while
    // the current epilogue runs
    float2 v[32];
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = __ldcs(Zrow + 32 * a);

    for (int j = 0; j < Kp; ++j) {
        __syncthreads();  // previous epilogue done with s_row (and s_tw ready on j = 0)
        {
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
        }
        __syncthreads();
        if (j + 1 < Kp) {
            const float2* Zn = Zrow + (int64_t)(j + 1) * zpair;
#pragma unroll
            for (int a = 0; a < 32; ++a) v[a] = __ldcs(Zn + 32 * a);
        }

        const bool has_odd = (2 * j + 1) < K;
        float2* J0 = J ? J + ((int64_t)b * K + 2 * j) * I : nullptr;
        float2* J1 = (J && has_odd) ? J + ((int64_t)b * K + 2 * j + 1) * I : nullptr;
        float* E0 = E ? E + ((int64_t)b * K + 2 * j) * I : nullptr;
        float* E1 = (E && has_odd) ? E + ((int64_t)b * K + 2 * j + 1) * I : nullptr;
#pragma unroll 4
        for (int it = 0; it < npos; ++it) {
            // position (slot offset, column) of k and of its partner nf - k
            int o1, c1, o2, c2, r1, r2;
            if (!self) {
                c1 = k2_0 + STEP * it;
                o1 = offL; r1 = rowL;
                o2 = offM; r2 = rowM; c2 = kRowLen - 1 - c1;
            } else if (it <= NIT / 2) {  // row 0, k2 in [0, 512]
                c1 = k2_0 + STEP * it;
                o1 = offL; r1 = 0;
                o2 = offL; r2 = 0; c2 = (kRowLen - c1) & (kRowLen - 1);
                if (c1 > kRowLen / 2) continue;
            } else {                     // row n1/2, k2 in [0, 512)
                c1 = k2_0 + STEP * (it - NIT / 2 - 1);
                o1 = offM; r1 = rowM;
                o2 = offM; r2 = rowM; c2 = kRowLen - 1 - c1;
            }
            const int kk1 = r1 + n1 * c1;
            const int kk2 = r2 + n1 * c2;
            const int i1 = (kk1 < half ? kk1 : kk1 - nf) + i_c;
            const int i2 = (kk2 < half ? kk2 : kk2 - nf) + i_c;
            const bool v1 = (unsigned)i1 < (unsigned)I;
            const bool v2 = (unsigned)i2 < (unsigned)I && kk2 != kk1;
            if (!v1 && !v2) continue;
            const float2 A = s_row[o1 + c1];
            const float2 Bc = s_row[o2 + c2];
            float2 sd;
            if (v1) {
                sd = __ldg(deconv + i1);
            } else {
                sd = __ldg(deconv + i2);
                sd.y = -sd.y;
            }
            // X_even = (A + conj(B)) / 2 ; X_odd = (A - conj(B)) / (2i)
            const float2 j0 = cmulf(make_float2(0.5f * (A.x + Bc.x), 0.5f * (A.y - Bc.y)), sd);
            const float p0 = j0.x * j0.x + j0.y * j0.y;
            if (v1) {
                if (J0) __stcs(J0 + i1, j0);
                if (E0) __stcs(E0 + i1, p0);
            }
            if (v2) {
                if (J0) __stcs(J0 + i2, make_float2(j0.x, -j0.y));
                if (E0) __stcs(E0 + i2, p0);
            }
            float pp = p0;
            if (has_odd) {
                const float2 j1 = cmulf(make_float2(0.5f * (A.y + Bc.y), -0.5f * (A.x - Bc.x)), sd);
                const float p1 = j1.x * j1.x + j1.y * j1.y;
                if (v1) {
                    if (J1) __stcs(J1 + i1, j1);
                    if (E1) __stcs(E1 + i1, p1);
                }
                if (v2) {
                    if (J1) __stcs(J1 + i2, make_float2(j1.x, -j1.y));
                    if (E1) __stcs(E1 + i2, p1);
                }
                pp += p1;
            }
            pacc[it * NT] += pp;
        }
    }
    if (Pout) {
        const float invK = 1.0f / (float)K;
        float* Pb = Pout + (int64_t)b * I;
        for (int it = 0; it < npos; ++it) {
            int c1, c2, r1, r2;
            if (!self) {
                c1 = k2_0 + STEP * it; r1 = rowL; r2 = rowM; c2 = kRowLen - 1 - c1;
            } else if (it <= NIT / 2) {
                c1 = k2_0 + STEP * it; r1 = 0; r2 = 0; c2 = (kRowLen - c1) & (kRowLen - 1);
                if (c1 > kRowLen / 2) continue;
            } else {
                c1 = k2_0 + STEP * (it - NIT / 2 - 1); r1 = rowM; r2 = rowM; c2 = kRowLen - 1 - c1;
            }
            const int kk1 = r1 + n1 * c1;
            const int kk2 = r2 + n1 * c2;
            const int i1 = (kk1 < half ? kk1 : kk1 - nf) + i_c;
            const int i2 = (kk2 < half ? kk2 : kk2 - nf) + i_c;
            const float pv = pacc[it * NT] * invK;
            if ((unsigned)i1 < (unsigned)I) __stcs(Pb + i1, pv);
            if ((unsigned)i2 < (unsigned)I && kk2 != kk1) __stcs(Pb + i2, pv);
        }
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
    M2_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
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
m2_status launch_rows_fast(m2nufft_plan_s* p, int nb, cudaStream_t st, const Tw32& tw, float2* J, float* E,
                           float* P) {
    const Geometry& g = p->g;
    const size_t smem = sizeof(float2) * ((size_t)kRowLen + (size_t)2 * R * kRowPad) +
                        sizeof(float) * (size_t)(kRowLen / 64 + 1) * 64 * R;  // P-hat accumulators [NIT + 1][NT]
    auto kern = rows_fast_kernel<R>;
    M2_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)(g.n1 / (2 * R)), (unsigned)nb);
    kern<<<grid, 64 * R, smem, st>>>(reinterpret_cast<const float2*>(p->d_Z), (int)g.n1, g.kp, g.K, (int)g.I,
                                     (int)g.i_c, (int)g.nf, reinterpret_cast<const float2*>(p->d_tw1024), tw,
                                     reinterpret_cast<const float2*>(p->d_deconv), J, E, P);
    M2_CUDA_TRY(cudaGetLastError());
    return M2_OK;
}

}  // namespace

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

    mark(p, 2, 0, st);
    {
        int R = 1;  // low rows per CTA: largest power of two <= 4 dividing n1 / 2
        while (R < kRowsR && (g.n1 / 2) % (R * 2) == 0) R *= 2;
        if (R == 8) M2_TRY(launch_rows_fast<8>(p, nb, st, tw, J, E, P));
        else if (R == 4) M2_TRY(launch_rows_fast<4>(p, nb, st, tw, J, E, P));
        else if (R == 2) M2_TRY(launch_rows_fast<2>(p, nb, st, tw, J, E, P));
        else M2_TRY(launch_rows_fast<1>(p, nb, st, tw, J, E, P));
    }
    mark(p, 2, 1, st);
    return M2_OK;
}

}  // namespace m2
