// 3PCF monopole by triple connection coefficients: Eq. (3pcfddd), Eq. (2-fold-density),
// Eq. (3PCF-ddd-monopole), Eq. (con-coeff), Eq. (DDD-vector-product), for the centred
// order-p B-spline basis of the scatter.
//
//   DDD(b1, b2) = (1/N^3) sum_l delta_l sum_{a,b} Gamma_{a,b} f_b1(l + a) f_b2(l + b),
//   Gamma_{a,b} = int phi(u) phi(u - a) phi(u - b) du,
//
// with f_b the l = 0 shell-filtered coefficients.  Summed over l this is the box integral
// (1/N^3) int D F_b1 F_b2 du of the three spline fields D = sum_l delta_l phi(u - l) and
// F_b = sum_l f_b(l) phi(u - l).  Between knots (integers for even p, half-integers for
// odd p) the integrand is a polynomial of degree 3(p - 1) along each axis, so a Gauss-
// Legendre rule of n_g = (3p - 1) / 2 points per axis and knot cell integrates it exactly:
// at order 4 the 37^3-term stencil becomes 125 samples per cell, and a spline field at the
// sample t_g of cell c is a p-tap filter along each axis, sum_j B_g[j] f(c + j0 + j).
//
// For every sample pair (g_z, g_y):
//   k_ddd_filter_yz: Y_f = the y and z filters of every field (delta and the shell fields),
//                    separable through shared memory;
//   k_ddd_gram     : down each (y, z) column, the x filters at every g_x (each field once per
//                    cell, from a sliding window of p x-taps in registers, shared through
//                    shared memory), then the weighted Gram sum_gx w_g D F_b1 F_b2 on 8 x 8 bin
//                    tiles, in float32 over one column (N cells x n_g samples), then float64.
//                    Up to 16 bins: two warps, each a diagonal tile and half of the off-
//                    diagonal one (three warps of one tile each, or one warp for up to 8 bins);
//                    more bins: one warp per pair of 8-bin blocks, the fields named by slot.
#include "kernels.h"

#include <algorithm>

namespace hermes {

namespace {

// Tiles of T y x T z outputs of one (field, x) plane (T = 64, or N below 64): the
// (T + P - 1)^2 inputs (periodic) staged once in shared memory by unrolled loads (several in
// flight per thread), filtered along z into a second stage, then along y.  Each filter step
// gives a thread a run of C outputs (C = T / 4) along its axis from a register window of
// C + P - 1 stage values, about 1.2 shared loads per output; the odd row pitches put the 32
// rows (z step) or columns (y step) of a warp on distinct banks.
template <int P, int T>
__global__ void __launch_bounds__(256) k_ddd_filter_yz(const float* __restrict__ in, float* __restrict__ out,
                                                       int lgN, const __grid_constant__ DddYZ tp) {
    constexpr int R = T + P - 1;
    constexpr int PIN = R | 1, PZ = T | 1;  // odd pitches
    constexpr int C = T / 4, NCH = 4;       // run length and runs per row / column
    constexpr int LOADS = (R * R + 255) / 256;
    constexpr int lgT = T == 64 ? 6 : (T == 32 ? 5 : 4);
    __shared__ float s_in[R][PIN];
    __shared__ float s_z[R][PZ];
    const int N = 1 << lgN, msk = N - 1;
    const int nt = N >> lgT;
    const size_t blk = blockIdx.x;
    const int tz = (int)(blk % nt), ty = (int)((blk / nt) % nt);
    const size_t plane = blk / ((size_t)nt * nt);  // field * N + x
    const int y0 = ty * T, z0 = tz * T;
    const float* src = in + (plane << (2 * lgN));
    float v[LOADS];
#pragma unroll
    for (int k = 0; k < LOADS; ++k) {
        const int e = threadIdx.x + k * 256;
        const int r = e / R, c = e - r * R;
        v[k] = (e < R * R) ? __ldg(src + ((size_t)((y0 + tp.j0 + r) & msk) << lgN) + ((z0 + tp.j0 + c) & msk)) : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < LOADS; ++k) {
        const int e = threadIdx.x + k * 256;
        const int r = e / R, c = e - r * R;
        if (e < R * R) s_in[r][c] = v[k];
    }
    __syncthreads();
    // along z: run (r, ch) = outputs ch*C .. ch*C + C - 1 of stage row r; consecutive threads, consecutive rows
    for (int e = threadIdx.x; e < R * NCH; e += 256) {
        const int r = e % R, ch = e / R;
        float w[C + P - 1];
#pragma unroll
        for (int q = 0; q < C + P - 1; ++q) w[q] = s_in[r][ch * C + q];
#pragma unroll
        for (int q = 0; q < C; ++q) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j) acc = fmaf(tp.bz[j], w[q + j], acc);
            s_z[r][ch * C + q] = acc;
        }
    }
    __syncthreads();
    // along y: run (c, ch) = output rows ch*C .. ch*C + C - 1 of column c; consecutive threads, consecutive columns
    float* dst = out + (plane << (2 * lgN));
    for (int e = threadIdx.x; e < T * NCH; e += 256) {
        const int c = e % T, ch = e / T;
        float w[C + P - 1];
#pragma unroll
        for (int q = 0; q < C + P - 1; ++q) w[q] = s_z[ch * C + q][c];
#pragma unroll
        for (int q = 0; q < C; ++q) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < P; ++j) acc = fmaf(tp.by[j], w[q + j], acc);
            dst[((size_t)(y0 + ch * C + q) << lgN) + z0 + c] = acc;
        }
    }
}

// Down 32 (y, z) columns per task, for x = 0 .. N-1: warp w x-filters field slots w, w + nw,
// ... (delta, the row block's bins, the column block's) at every sample g_x from its sliding
// windows of P taps and stages the values in shared memory (double-buffered, one barrier per
// cell); then warp w adds w_gx D F_b1 F_b2 into its tile of the Gram.  Empty slots stay zero.
template <int P, int NW>
__global__ void __launch_bounds__(32 * NW, NW == 3 ? 4 : (NW == 2 ? 6 : 8))
    k_ddd_gram(const float* __restrict__ Y, int lgN, const __grid_constant__ DddTaps tp, double* __restrict__ part) {
    constexpr int NG = ddd_samples(P), FPW = (17 + NW - 1) / NW;  // slots filtered per warp, at most
    constexpr int nw = NW;
    __shared__ float s_v[2][NG][17][32];
    const int N = 1 << lgN, msk = N - 1, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t n3 = (size_t)1 << (3 * lgN);
    constexpr int nf = 17;
    for (int e = threadIdx.x; e < 2 * NG * 17 * 32; e += blockDim.x) (&s_v[0][0][0][0])[e] = 0.0f;
    // 0 (rows, rows), 1 (rows, columns), 2 (columns, columns).  Two warps: warp w takes the
    // diagonal tile 2w and the columns 4w .. 4w + 3 of tile 1 (equal work per warp).
    const int tile = nw == 1 ? tp.tile0 : (nw == 2 ? 2 * w : w);
    const int slot_out = nw == 1 ? 0 : tile;      // where the tile's entries are written
    const int r0 = tile == 2 ? 8 : 0, c0 = tile == 0 ? 0 : 8;
    const bool diag = tile != 1;
    // the Y offsets of the slots this warp filters (-1: empty), fixed for the kernel
    long long foff[FPW];
#pragma unroll
    for (int k = 0; k < FPW; ++k) {
        const int f = w + k * nw;
        const int fi = f < nf ? tp.fld[f] : -1;
        foff[k] = fi >= 0 ? (long long)fi * (long long)n3 : -1;
    }
    double d0 = 0.0, d1 = 0.0, e0 = 0.0, e1 = 0.0;  // e: the half of tile 1 (two warps)
    int buf = 0;
    const int ntask = (N * N) >> 5;
    __syncthreads();
    for (int task = blockIdx.x; task < ntask; task += gridDim.x) {
        const float* col = Y + ((size_t)task << 5) + lane;
        float t[FPW][P];
#pragma unroll
        for (int k = 0; k < FPW; ++k) {
#pragma unroll
            for (int j = 0; j < P; ++j)
                t[k][j] = foff[k] >= 0 ? __ldg(col + foff[k] + ((size_t)((tp.j0 + j) & msk) << (2 * lgN))) : 0.0f;
        }
        float acc[64];
#pragma unroll
        for (int k = 0; k < 64; ++k) acc[k] = 0.0f;
        float acc2[NW == 2 ? 32 : 1];
#pragma unroll
        for (int k = 0; k < (NW == 2 ? 32 : 1); ++k) acc2[k] = 0.0f;
        for (int x = 0; x < N; ++x) {
            float nxt[FPW];  // the tap entering each window at x + 1, in flight during this cell
            const size_t xn = (size_t)((x + 1 + tp.j0 + P - 1) & msk) << (2 * lgN);
#pragma unroll
            for (int k = 0; k < FPW; ++k) nxt[k] = foff[k] >= 0 ? __ldg(col + foff[k] + xn) : 0.0f;
#pragma unroll
            for (int k = 0; k < FPW; ++k) {
                const int f = w + k * nw;
                if (foff[k] >= 0) {
#pragma unroll
                    for (int g = 0; g < NG; ++g) {
                        float v = 0.0f;
#pragma unroll
                        for (int j = 0; j < P; ++j) v = fmaf(tp.bx[g][j], t[k][j], v);
                        s_v[buf][g][f][lane] = v;
                    }
                }
            }
            __syncthreads();
#pragma unroll 1
            for (int g = 0; g < NG; ++g) {
                const float h = tp.wx[g] * s_v[buf][g][0][lane];
                float vr[8];
#pragma unroll
                for (int a2 = 0; a2 < 8; ++a2) vr[a2] = h * s_v[buf][g][1 + r0 + a2][lane];
                if (diag) {
#pragma unroll
                    for (int a2 = 0; a2 < 8; ++a2) {
#pragma unroll
                        for (int b2 = a2; b2 < 8; ++b2)
                            acc[a2 * 8 + b2] = fmaf(vr[a2], s_v[buf][g][1 + r0 + b2][lane], acc[a2 * 8 + b2]);
                    }
                    if constexpr (NW == 2) {  // rows 1..8 x columns 9 + 4w .. 12 + 4w
                        float vcb[4];
#pragma unroll
                        for (int b2 = 0; b2 < 4; ++b2) vcb[b2] = s_v[buf][g][9 + 4 * w + b2][lane];
#pragma unroll
                        for (int a2 = 0; a2 < 8; ++a2) {
                            const float hr = w == 0 ? vr[a2] : h * s_v[buf][g][1 + a2][lane];
#pragma unroll
                            for (int b2 = 0; b2 < 4; ++b2) acc2[a2 * 4 + b2] = fmaf(hr, vcb[b2], acc2[a2 * 4 + b2]);
                        }
                    }
                } else {
                    float vc[8];
#pragma unroll
                    for (int b2 = 0; b2 < 8; ++b2) vc[b2] = s_v[buf][g][1 + c0 + b2][lane];
#pragma unroll
                    for (int a2 = 0; a2 < 8; ++a2) {
#pragma unroll
                        for (int b2 = 0; b2 < 8; ++b2) acc[a2 * 8 + b2] = fmaf(vr[a2], vc[b2], acc[a2 * 8 + b2]);
                    }
                }
            }
            buf ^= 1;
#pragma unroll
            for (int k = 0; k < FPW; ++k) {
#pragma unroll
                for (int j = 0; j + 1 < P; ++j) t[k][j] = t[k][j + 1];
                t[k][P - 1] = nxt[k];
            }
        }
        // the column's float32 sums, summed over the warp, into float64 (entry k on lane k % 32);
        // diagonal tiles leave the lower triangle at zero
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            float sum = acc[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (lane == (k & 31)) {
                if (k < 32) d0 += (double)sum;
                else d1 += (double)sum;
            }
        }
        if constexpr (NW == 2) {  // entry 8 a + 4 w + b of tile 1
#pragma unroll
            for (int k2 = 0; k2 < 32; ++k2) {
                float sum = acc2[k2];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                const int k = 8 * (k2 / 4) + 4 * w + (k2 % 4);
                if (lane == (k & 31)) {
                    if (k < 32) e0 += (double)sum;
                    else e1 += (double)sum;
                }
            }
        }
    }
    // accumulate over the (g_z, g_y) launches: each (block, tile, entry) has one owner
    double* row = part + ((size_t)blockIdx.x * 3 + slot_out) * 64;
    row[lane] += d0 * tp.wyz;
    row[32 + lane] += d1 * tp.wyz;
    if (NW == 2 && ((lane & 7) >> 2) == w) {  // entries lane and lane + 32 of tile 1 are this warp's
        double* r1 = part + ((size_t)blockIdx.x * 3 + 1) * 64;
        r1[lane] += e0 * tp.wyz;
        r1[32 + lane] += e1 * tp.wyz;
    }
}

int ilog2i(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

int sm_count_ddd() {
    static int n = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || v <= 0) {
            cudaGetLastError();
            return 148;
        }
        return v;
    }();
    return n;
}

}  // namespace

int ddd_gram_blocks(int N, int nw) {
    // the blocks per SM the two forms are compiled for (3 warps: 4, one warp: 8); never more
    // blocks than 32-column tasks
    return std::max(1, std::min((nw == 1 ? 8 : (nw == 2 ? 6 : 4)) * sm_count_ddd(), (N * N) / 32));
}

cudaError_t launch_ddd_filter_yz(int N, int p, const float* in, float* out, int nf, const DddYZ& tp,
                                 cudaStream_t st, const Tracer& tr) {
    if (N < 16) return cudaErrorInvalidValue;
    const int lgN = ilog2i(N), lgT = std::min(lgN, 6);
    const size_t nt = (size_t)N >> lgT;
    const size_t nblk = (size_t)nf * N * nt * nt;  // (field, x) planes x y tiles x z tiles
    if (nblk > 0x7fffffffULL) return cudaErrorInvalidValue;
    tr(K_DDD_FILTER, 0, st);
    switch (p) {
#define C(P)                                                                                    \
    case P:                                                                                     \
        if (lgT == 6) k_ddd_filter_yz<P, 64><<<(unsigned)nblk, 256, 0, st>>>(in, out, lgN, tp);   \
        else if (lgT == 5) k_ddd_filter_yz<P, 32><<<(unsigned)nblk, 256, 0, st>>>(in, out, lgN, tp); \
        else k_ddd_filter_yz<P, 16><<<(unsigned)nblk, 256, 0, st>>>(in, out, lgN, tp);            \
        break;
        C(1) C(2) C(3) C(4)
#undef C
        default: return cudaErrorInvalidValue;
    }
    tr(K_DDD_FILTER, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_ddd_gram(int N, int p, const float* Y, int nw, const DddTaps& tp, double* part, cudaStream_t st,
                            const Tracer& tr) {
    if (nw < 1 || nw > 3 || N < 16 || tp.fld[0] < 0) return cudaErrorInvalidValue;
    const int lgN = ilog2i(N);
    const int nblk = ddd_gram_blocks(N, nw);
    tr(K_DDD_GRAM, 0, st);
    switch (p) {
#define C(P)                                                                      \
    case P:                                                                       \
        if (nw == 1) k_ddd_gram<P, 1><<<nblk, 32, 0, st>>>(Y, lgN, tp, part);      \
        else if (nw == 2) k_ddd_gram<P, 2><<<nblk, 64, 0, st>>>(Y, lgN, tp, part); \
        else k_ddd_gram<P, 3><<<nblk, 96, 0, st>>>(Y, lgN, tp, part);             \
        break;
        C(1) C(2) C(3) C(4)
#undef C
        default: return cudaErrorInvalidValue;
    }
    tr(K_DDD_GRAM, 1, st);
    return cudaGetLastError();
}

}  // namespace hermes
