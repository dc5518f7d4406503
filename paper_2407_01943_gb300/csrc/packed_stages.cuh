// Device-side stages of the packed FP32 exec path, shared by the four
// stand-alone kernels (fast.cu) and the persistent pipelined kernel (pipe.cu).
//
// Mathematics (Sec. 3.2, Eq. eigencoefficients and Eq.
// power_spectrum_estimator, evaluated by a type-1 nonuniform FFT):
//   * two real tapers share one complex FFT: the spread grid of taper pair j is
//     g_{2j} + i g_{2j+1}; both grids are real, so their transforms follow from
//     the packed transform Zp at k and nf - k:
//         X_{2j}[k]   = (Zp[k] + conj(Zp[nf-k])) / 2
//         X_{2j+1}[k] = (Zp[k] - conj(Zp[nf-k])) / (2i);
//   * four-step FFT nf = n1 * 1024 with the spread support in the first `rows`
//     rows: column DFTs per coset k1 = r + C q (C = n1/F) by folding the inputs
//     modulo F and one F-point register FFT, then 1024-point row FFTs (one warp
//     per row, 32 x 32 in registers, one padded shared-memory transpose),
//     written transposed (Xt[k2][k1]);
//   * epilogue: one thread per output pair (m, -m): J(-m) = conj J(m) since
//     both tapers are real and the deconvolution factor satisfies
//     s(-m) = conj s(m); P-hat summed over the pairs in registers.
// Intermediates (g, Z, Xt) are read with ld.global.cg (L2, not L1), so stages
// may consume data written by other CTAs of the same kernel.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace m2 {
namespace packed {

constexpr int kRowLen = 1024;  // n2
constexpr int kRowPad = 1060;  // per-warp transpose / row buffer: >= 32 x 33 (padded transpose)
constexpr int kColWarps = 4;   // warps per 32-column group of the column pass
constexpr int kRowsPerGroup = 8;  // rows per row-FFT work item (one warp each)

struct Tw32 {
    float2 w[16];  // exp(-i 2 pi e / 32), e < 16
};

// Complex product and squared magnitude with the rounding spelled out (one product rounded, the
// other fused), so that every kernel that inlines a stage -- whatever the compiler would contract
// there -- computes the same bits.
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float norm2f(float2 a) { return __fmaf_rn(a.x, a.x, __fmul_rn(a.y, a.y)); }

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

// Plan data the stages read (one plan; device pointers).
struct __align__(16) Ctx {
    const int32_t* pt_src;
    const int32_t* pt_cell;
    const float* pt_off;
    const float* taper;  // [K][P] real
    int64_t P;
    const int32_t* tile_pb;
    const int32_t* tile_pe;
    int N, K, Kp, w;
    float two_over_w, beta;
    int64_t Lg;          // spread cells per pair = rows * 1024
    int rows, n1;
    int I, i_c, nf, k2max;
    int F;                 // coset FFT length of the column pass (largest power of two <= 32 dividing n1)
    int cgw;               // persistent kernel: warps per 32-column group of the column pass (1, 2 or 4)
    int cm;                // persistent kernel: column passes (8 / cgw groups of 32 columns each) per item
    const float2* tw_n1;   // [n1]
    const float2* colT;    // [F][1024]
    const float2* colB;    // [C][1024]
    const float2* tw1024;  // [32][32]: [cc][l] = W_1024^{cc l}
    const float2* deconv;  // [I]
    const float* wsum;     // [K] W_k^0(0) = sum_n w_k(t_n) (F-statistic), or NULL
    float wq;              // sum_k W_k^0(0)^2
};

// Drop a dead 128-byte line of an intermediate from L2 without writing it back (its contents
// become undefined; the next writer of the workspace overwrites it before anyone reads it).
// p: 128-byte aligned.
__device__ __forceinline__ void discard_l2(const void* p) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

// Load of an intermediate written earlier: kStream = streaming (evict-first) for the
// stand-alone kernels, where each value is read once; otherwise L2-only (.cg), which
// is coherent with stores made by other CTAs of the same kernel.
template <bool kStream>
__device__ __forceinline__ float2 ld_inter(const float2* p) {
    if (kStream) return __ldcs(p);
    return __ldcg(p);
}

// ---------------------------------------------------------------------------
// spread tiles [tile0, tile0 + nt) (256 cells each, nt <= NT) of one signal:
//   g[j][c] = sum_n (u_{2j}[n] + i u_{2j+1}[n]) x[n] phi(c - u_n)
// Thread = cell tile0 * 256 + 256 u + threadIdx.x for u < nt.  The points whose
// windows meet the tiles are staged in chunks; every cell adds its points in
// ascending point order, so the result does not depend on NT.
// blockDim = kSpreadTile; smem >= spread_smem_bytes(KP).
// ---------------------------------------------------------------------------
template <int KP, int NT>
__device__ __forceinline__ void spread_tiles(const Ctx& c, const float* __restrict__ xb, int tile0, int nt,
                                             float2* __restrict__ gb, unsigned char* smem) {
    int32_t* s_cell = reinterpret_cast<int32_t*>(smem);
    float* s_off = reinterpret_cast<float*>(smem + 4 * kSpreadChunk);
    float2* s_val = reinterpret_cast<float2*>(smem + 8 * kSpreadChunk);  // [KP][chunk]
    const int64_t cell0 = (int64_t)tile0 * kSpreadTile + threadIdx.x;
    const int pb = c.tile_pb[tile0], pe = c.tile_pe[tile0 + nt - 1];
    float2 acc[NT][KP];
#pragma unroll
    for (int u = 0; u < NT; ++u)
#pragma unroll
        for (int j = 0; j < KP; ++j) acc[u][j] = make_float2(0.f, 0.f);
    for (int q0 = pb; q0 < pe; q0 += kSpreadChunk) {
        const int n = min(kSpreadChunk, pe - q0);
        __syncthreads();
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int p = q0 + t;
            s_cell[t] = c.pt_cell[p];
            s_off[t] = c.pt_off[p];
            const float xv = xb[c.pt_src[p]];
#pragma unroll
            for (int j = 0; j < KP; ++j) {
                float2 v = make_float2(0.f, 0.f);
                if (2 * j < c.K) v.x = c.taper[(int64_t)(2 * j) * c.P + p] * xv;
                if (2 * j + 1 < c.K) v.y = c.taper[(int64_t)(2 * j + 1) * c.P + p] * xv;
                s_val[j * kSpreadChunk + t] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < NT; ++u) {
            const int64_t cell = cell0 + (int64_t)u * kSpreadTile;
            if (u < nt && cell < c.Lg) {
                const int ci = (int)cell;
                int lo = 0, hi = n;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (s_cell[mid] + c.w <= ci) lo = mid + 1; else hi = mid;
                }
                for (int t = lo; t < n && s_cell[t] <= ci; ++t) {
                    const float z = s_off[t] + (float)(ci - s_cell[t]);
                    const float a = z * c.two_over_w;
                    const float phi = expf(c.beta * (sqrtf(fmaxf(0.f, 1.f - a * a)) - 1.f));
#pragma unroll
                    for (int j = 0; j < KP; ++j) {
                        const float2 v = s_val[j * kSpreadChunk + t];
                        acc[u][j].x += v.x * phi;
                        acc[u][j].y += v.y * phi;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < NT; ++u) {
        const int64_t cell = cell0 + (int64_t)u * kSpreadTile;
        if (u < nt && cell < c.Lg) {
#pragma unroll
            for (int j = 0; j < KP; ++j)
                if (j < c.Kp) gb[(int64_t)j * c.Lg + cell] = acc[u][j];
        }
    }
    __syncthreads();  // smem reuse by the next stage of this CTA
}

template <int KP>
__device__ __forceinline__ void spread_tile(const Ctx& c, const float* __restrict__ xb, int tile,
                                            float2* __restrict__ gb, unsigned char* smem) {
    spread_tiles<KP, 1>(c, xb, tile, 1, gb, smem);
}

// ---------------------------------------------------------------------------
// spread one tile for SB signals of one plan at once (signals b0 .. b0 + nsb - 1,
// x and g strided by N and Kp * Lg): the point records, tapers and window
// searches are shared by all signals of a plan, so they are staged once per
// tile; per signal the arithmetic and its order are those of spread_tiles, so
// each signal's grid is bit-identical to spreading it alone.
// smem >= spread_multi_smem_bytes(KP, SB).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr size_t spread_multi_smem_bytes(int KP, int SB) {
    return (size_t)8 * kSpreadChunk + (size_t)KP * kSpreadChunk * 8 + (size_t)SB * kSpreadChunk * 4;
}

template <int KP, int SB>
__device__ __forceinline__ void spread_tile_multi(const Ctx& c, const float* __restrict__ x, int nsb, int tile,
                                                  float2* __restrict__ g, unsigned char* smem) {
    int32_t* s_cell = reinterpret_cast<int32_t*>(smem);
    float* s_off = reinterpret_cast<float*>(smem + 4 * kSpreadChunk);
    float2* s_tap = reinterpret_cast<float2*>(smem + 8 * kSpreadChunk);                      // [KP][chunk]
    float* s_x = reinterpret_cast<float*>(smem + 8 * kSpreadChunk + KP * kSpreadChunk * 8);  // [SB][chunk]
    const int64_t cell = (int64_t)tile * kSpreadTile + threadIdx.x;
    const int pb = c.tile_pb[tile], pe = c.tile_pe[tile];
    float2 acc[SB][KP];
#pragma unroll
    for (int b = 0; b < SB; ++b)
#pragma unroll
        for (int j = 0; j < KP; ++j) acc[b][j] = make_float2(0.f, 0.f);
    for (int q0 = pb; q0 < pe; q0 += kSpreadChunk) {
        const int n = min(kSpreadChunk, pe - q0);
        __syncthreads();
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int p = q0 + t;
            s_cell[t] = c.pt_cell[p];
            s_off[t] = c.pt_off[p];
            const int src = c.pt_src[p];
#pragma unroll
            for (int b = 0; b < SB; ++b) s_x[b * kSpreadChunk + t] = b < nsb ? x[(int64_t)b * c.N + src] : 0.f;
#pragma unroll
            for (int j = 0; j < KP; ++j) {
                float2 v = make_float2(0.f, 0.f);
                if (2 * j < c.K) v.x = c.taper[(int64_t)(2 * j) * c.P + p];
                if (2 * j + 1 < c.K) v.y = c.taper[(int64_t)(2 * j + 1) * c.P + p];
                s_tap[j * kSpreadChunk + t] = v;
            }
        }
        __syncthreads();
        if (cell < c.Lg) {
            const int ci = (int)cell;
            int lo = 0, hi = n;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_cell[mid] + c.w <= ci) lo = mid + 1; else hi = mid;
            }
            for (int t = lo; t < n && s_cell[t] <= ci; ++t) {
                const float z = s_off[t] + (float)(ci - s_cell[t]);
                const float a = z * c.two_over_w;
                const float phi = expf(c.beta * (sqrtf(fmaxf(0.f, 1.f - a * a)) - 1.f));
#pragma unroll
                for (int b = 0; b < SB; ++b) {
                    const float xv = s_x[b * kSpreadChunk + t];
#pragma unroll
                    for (int j = 0; j < KP; ++j) {
                        const float2 tp = s_tap[j * kSpreadChunk + t];
                        const float vx = tp.x * xv, vy = tp.y * xv;  // the tapered sample, rounded as when spread alone
                        acc[b][j].x += vx * phi;
                        acc[b][j].y += vy * phi;
                    }
                }
            }
        }
    }
    if (cell < c.Lg) {
#pragma unroll
        for (int b = 0; b < SB; ++b)
            if (b < nsb) {
#pragma unroll
                for (int j = 0; j < KP; ++j)
                    if (j < c.Kp) g[((int64_t)b * c.Kp + j) * c.Lg + cell] = acc[b][j];
            }
    }
}

__host__ __device__ constexpr size_t spread_smem_bytes(int KP) { return (size_t)8 * kSpreadChunk + (size_t)KP * kSpreadChunk * 8; }

// ---------------------------------------------------------------------------
// column pass for 32 columns starting at colbase, done by a group of gw warps
// (gwarp = this warp's index in the group); every warp of the CTA calls this
// once per pass, so the CTA-wide barriers line up:
//   Z[k1][l2] = W_nf^{l2 k1} sum_{l1 < rows} g[l1][l2] W_n1^{l1 k1}
// The group's warps share the C = n1 / F cosets.  s_tw: [n1] twiddles W_n1^q,
// filled by the caller before the call (the first barrier inside publishes
// them).  smem: this group's [rows][32] + [F][32].
// ---------------------------------------------------------------------------
template <int F>
__device__ __forceinline__ void cols_group(const Ctx& c, const Tw32& tw, const float2* __restrict__ gj,
                                           float2* __restrict__ Zj, int colbase, int gwarp, int gw,
                                           const float2* s_tw, float2* smem) {
    float2* s_in = smem;                // [rows][32]
    float2* s_T = s_in + c.rows * 32;   // [F][32]
    const int lane = threadIdx.x & 31;
    const int l2 = colbase + lane;
    const int n1 = c.n1, rows = c.rows;
    const int C = n1 / F;
    for (int l1 = gwarp; l1 < rows; l1 += gw) s_in[l1 * 32 + lane] = __ldcg(gj + (int64_t)l1 * kRowLen + l2);
    for (int q = gwarp; q < F; q += gw) s_T[q * 32 + lane] = __ldg(c.colT + q * kRowLen + l2);
    __syncthreads();
    const int nfold = (rows + F - 1) / F;
    for (int r = gwarp; r < C; r += gw) {
        const float2 base = __ldg(c.colB + (int64_t)r * kRowLen + l2);
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
            Zj[(int64_t)k1 * kRowLen + l2] = cmulf(v[brev(q, ilog2c(F))], t);
        }
    }
    __syncthreads();  // smem reuse
}

// shared memory of one column group (float2 units, excluding the [n1] twiddles)
__host__ __device__ inline size_t cols_group_f2(int rows, int F) { return (size_t)rows * 32 + (size_t)F * 32; }

// One 1024-point row FFT by one warp: S[k2] = sum_{l2} Zr[l2] W_1024^{l2 k2} in natural
// order; S holds >= 32 x 33 float2 (the padded transpose between the two radix-32 passes).
template <bool kStream>
__device__ __forceinline__ void rowfft_one(const Ctx& c, const Tw32& tw, const float2* __restrict__ Zr,
                                           float2* S) {
    const int lane = threadIdx.x & 31;
    float2 v[32];
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = ld_inter<kStream>(Zr + lane + 32 * a);
    fft_reg<32>(v, tw);  // over a for column b = lane: v[q] = Y[lane][brev(q)]
    // twiddle W_1024^{lane cc} from the (L1-resident) [cc][lane] table: 256 contiguous bytes per warp
    const float2* twl = c.tw1024 + lane;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        const int cc = brev(q, 5);
        S[cc * 33 + lane] = cmulf(v[q], __ldg(twl + 32 * cc));
    }
    __syncwarp();
    // stand-alone kernels: this warp was the row's only reader, and every lane's loads have been
    // consumed, so its 64 lines are dead (Zr is 8 KB aligned: Z rows are 1024 complex)
    if (kStream) {
        discard_l2(Zr + 32 * lane);
        discard_l2(Zr + 32 * lane + 16);
    }
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = S[lane * 33 + a];
    __syncwarp();
    fft_reg<32>(v, tw);  // over b for column cc = lane: v[q] = X[lane + 32 brev(q)]
#pragma unroll
    for (int q = 0; q < 32; ++q) S[lane + 32 * brev(q, 5)] = v[q];
}

// ---------------------------------------------------------------------------
// row FFTs of rows [r0, r0 + nr), nr <= R (warp w < nr = row r0 + w; the other
// warps only take part in the barriers), written transposed for the in-band
// columns k2 <= k2max and k2 >= 1023 - k2max only:
//   Xt[k2][k1] = sum_{l2} Z[k1][l2] W_1024^{l2 k2}
// Called by all 32 R threads of the CTA.  smem (float2): R * kRowPad.
// ---------------------------------------------------------------------------
template <int R, bool kStream>
__device__ __forceinline__ void rowfft_rows(const Ctx& c, const Tw32& tw, const float2* __restrict__ Zj,
                                            float2* __restrict__ Xtj, int r0, int nr, float2* smem) {
    constexpr int NT = 32 * R;
    float2* s_row = smem;  // [R][kRowPad]
    const int warp = threadIdx.x >> 5;
    if (warp < nr) rowfft_one<kStream>(c, tw, Zj + (int64_t)(r0 + warp) * kRowLen, s_row + warp * kRowPad);
    __syncthreads();
    // Xt[k2][r0 + rr] for rr < nr: consecutive threads take consecutive rows
    float2* Xb = Xtj + r0;
    const int nlo = c.k2max + 1;  // k2 in [0, nlo)
    const int nout = 2 * nlo;     // plus k2 in [1024 - nlo, 1024)
    const int n1 = c.n1;
    if (nr == R) {
#pragma unroll 4
        for (int e = threadIdx.x; e < R * nout; e += NT) {
            const int rr = e % R, q = e / R;
            const int k2 = q < nlo ? q : kRowLen - nout + q;
            Xb[(int64_t)k2 * n1 + rr] = s_row[rr * kRowPad + k2];
        }
    } else {
        for (int e = threadIdx.x; e < nr * nout; e += NT) {
            const int rr = e % nr, q = e / nr;
            const int k2 = q < nlo ? q : kRowLen - nout + q;
            Xb[(int64_t)k2 * n1 + rr] = s_row[rr * kRowPad + k2];
        }
    }
    __syncthreads();  // smem reuse
}

inline size_t rowfft_smem_bytes(int R) { return sizeof(float2) * (size_t)R * kRowPad; }

// ---------------------------------------------------------------------------
// epilogue for position k = k1 + n1 k2 (k2 <= k2max) and its partner nf - k:
// (n1 - k1, 1023 - k2), or (0, 1024 - k2) for k1 = 0.  Unpack each taper pair,
// deconvolve, write J and |J|^2 at m and -m, and the taper average P-hat.
// Xtb: [Kp][1024][n1]; J, E: [K][I]; P: [I] (this signal; NULL = not wanted).
// ---------------------------------------------------------------------------
// With kF, also Thomson's F-statistic (Sec. 3, Eq. f_stat) at m and -m (equal, since
// J_k(-m) = conj J_k(m) and W_k^0(0) is real):
//   C = sum_k J_k W_k / sum_k W_k^2,  F = |C|^2 (K - 1) sum_k W_k^2 / sum_k |J_k - C W_k|^2.
template <bool kStream, bool kF = false>
__device__ __forceinline__ void epi_position(const Ctx& c, const float2* __restrict__ Xtb, int k1, int k2,
                                             float2* __restrict__ J, float* __restrict__ E,
                                             float* __restrict__ Pout, float* __restrict__ Fout = nullptr) {
    const int n1 = c.n1, nf = c.nf, I = c.I, K = c.K;
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
    const int i1 = (kk1 < half ? kk1 : kk1 - nf) + c.i_c;
    const int i2 = (kk2 < half ? kk2 : kk2 - nf) + c.i_c;
    const bool v1 = (unsigned)i1 < (unsigned)I;
    const bool v2 = (unsigned)i2 < (unsigned)I && kk2 != kk1;
    if (!v1 && !v2) return;
    float2 sd;
    if (v1) {
        sd = __ldg(c.deconv + i1);
    } else {
        sd = __ldg(c.deconv + i2);
        sd.y = -sd.y;
    }
    const int64_t plane = (int64_t)n1 * kRowLen;
    const float2* X1 = Xtb + (int64_t)k2 * n1 + k1;
    const float2* X2 = Xtb + (int64_t)pk2 * n1 + pk1;
    const int Kp = c.Kp;
    float pacc = 0.f;
    constexpr int kMaxPairs = kF ? (kMaxK + 1) / 2 : 1;
    float2 jk[kMaxPairs][2];  // kF: J of every taper at m, for the residual of the line fit
    float2 csum = make_float2(0.f, 0.f);
    auto pair = [&](int j) {
        const float2 A = ld_inter<kStream>(X1 + (int64_t)j * plane);
        const float2 Bc = ld_inter<kStream>(X2 + (int64_t)j * plane);
        // X_even = (A + conj(B)) / 2 ; X_odd = (A - conj(B)) / (2i)
        const float2 j0 = cmulf(make_float2(0.5f * (A.x + Bc.x), 0.5f * (A.y - Bc.y)), sd);
        const float p0 = norm2f(j0);
        const int64_t o0 = (int64_t)(2 * j) * I;
        if (J) {
            if (v1) __stcs(J + o0 + i1, j0);
            if (v2) __stcs(J + o0 + i2, make_float2(j0.x, -j0.y));
        }
        if (E) {
            if (v1) __stcs(E + o0 + i1, p0);
            if (v2) __stcs(E + o0 + i2, p0);
        }
        pacc += p0;
        if (kF) {
            const float w0 = c.wsum[2 * j];
            jk[kF ? j : 0][0] = j0;
            csum.x += j0.x * w0;
            csum.y += j0.y * w0;
        }
        if (2 * j + 1 < K) {
            const float2 j1 = cmulf(make_float2(0.5f * (A.y + Bc.y), -0.5f * (A.x - Bc.x)), sd);
            if (kF) {
                const float w1 = c.wsum[2 * j + 1];
                jk[kF ? j : 0][1] = j1;
                csum.x += j1.x * w1;
                csum.y += j1.y * w1;
            }
            const float p1 = norm2f(j1);
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
    };
    if constexpr (kF) {
#pragma unroll
        for (int j = 0; j < kMaxPairs; ++j)
            if (j < Kp) pair(j);  // fully unrolled: jk stays in registers
    } else {
        for (int j = 0; j < Kp; ++j) pair(j);
    }
    if (Pout) {
        const float pv = pacc * (1.0f / (float)K);
        if (v1) __stcs(Pout + i1, pv);
        if (v2) __stcs(Pout + i2, pv);
    }
    if (kF && Fout) {
        const float2 ch = make_float2(csum.x / c.wq, csum.y / c.wq);  // line amplitude C at m
        float res = 0.f;
#pragma unroll
        for (int j = 0; j < kMaxPairs; ++j) {
            if (j >= Kp) break;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (2 * j + h < K) {
                    const float wk = c.wsum[2 * j + h];
                    const float rx = jk[j][h].x - ch.x * wk, ry = jk[j][h].y - ch.y * wk;
                    res += rx * rx + ry * ry;
                }
            }
        }
        const float fv = (ch.x * ch.x + ch.y * ch.y) * (float)(K - 1) * c.wq / res;
        if (v1) __stcs(Fout + i1, fv);
        if (v2) __stcs(Fout + i2, fv);
    }
}

// Twiddles exp(-i 2 pi e / 32), e < 16, for the register FFTs.
Tw32 make_tw32();

}  // namespace packed

// Stage context of a packed plan (host side; reads the plan's device buffers).
packed::Ctx packed_ctx(const m2nufft_plan_s* p);
// Positions on the m >= 0 side of the packed spectrum: k2 <= k2max.
int packed_k2max(const Geometry& g);

}  // namespace m2
