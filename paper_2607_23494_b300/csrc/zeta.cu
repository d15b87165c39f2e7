// 3PCF multipole path: harmonic shell fields and their weighted Gram product.
//
// For one (l, m >= 0) and a batch of S <= 16 radial bins b, the fields
//   a_{b lm} = iFFT[ delta^ K_{b lm} ],  K_{b lm} = 4 pi i^l <j_l>_b(k) Y_lm(k^) Phi^,
// (Eq. multipole-window and Eq. iFFT-multipoleSFC) are complex and have no
// Hermitian symmetry, so the inverse is a full complex-to-complex transform:
//   Z1 along x: read the half spectrum (the k_z < 0 half is conj(delta^(-n))),
//      multiply by K_{b lm} for every bin, inverse FFT, store;
//   Z2 along y;
//   Z3 along z for all bins of one (x, y) line, fused with the weighted Gram
//      G(b1,b2) += sum_z delta(z) Re(conj(a_b1(z)) a_b2(z))
//   so the filtered fields never return to HBM after the y pass.
// zeta_l = 1/(4 pi N^3) sum_x delta sum_{m=-l}^{l} conj(a_b1) a_b2 then equals
// (G_{l0} + 2 sum_{m>0} G_{lm}) / (4 pi N^9) on the unnormalised transforms,
// since a_{l,-m} = (-1)^m conj(a_{lm}) for a real field (Eq. 2-fold-translation,
// negative m recovered by conjugation as in Sec. 4.4).  For m = 0 the fields are real
// (K_{b l0}(-k) = conj K_{b l0}(k)), so two bins share one complex transform,
// a_{2f} + i a_{2f+1}, and the Gram takes their real and imaginary parts apart.
#include "kernels.h"
#include "fft_core.cuh"
#include "async_copy.cuh"

#include <cstdlib>

namespace hermes {

template <int N>
struct ZCfg {
    static constexpr int H = N / 2;
    static constexpr int W = (N >= 512) ? 8 : (N / 2 < 16 ? N / 2 : 16);
    static constexpr int TS = (N / 8) * W;
    static constexpr int T = N / 8;                       // threads per z line
    static constexpr int GB = (512 / T) < 16 ? (512 / T) : 16;  // bin lines per round
    static constexpr int ZT = GB * T;                     // z-pass threads
    static constexpr int NZS = ZT / 16;                   // z slices in the Gram phase
    static constexpr int ZPER = N / NZS;                  // z values per slice
    static constexpr int LPZ = LinePad<N>::value + 4;     // line stride: +8 words skew per line
    static constexpr size_t SMEM_X = (size_t)SmemStrided<W>::words(N) * sizeof(float2);
    // z pass: 16 padded bin lines, two delta lines and (N <= 512) a stage for the next line's bins
    static constexpr bool PREFETCH = N <= 512;
    static constexpr size_t SMEM_Z = (size_t)16 * LPZ * sizeof(float2) + (size_t)2 * N * sizeof(float) +
                                     (PREFETCH ? (size_t)16 * N * sizeof(float2) : 0);
};
static_assert(ZCfg<16>::ZPER >= 1 && ZCfg<1024>::NZS == 32, "z-pass layout");
static_assert(ZCfg<512>::GB <= 15 && ZCfg<1024>::GB <= 15, "one named barrier per z line group");

// As allow_smem in the inverse passes: the attribute is shared by every host thread, so it
// is always set to one value (220 KiB, next to at most 7 KiB of static arrays) rather than
// to the size of one launch (the x pass stages S-dependent tables).
template <class K>
static cudaError_t allow_smem_z(K kernel, size_t bytes) {
    constexpr size_t kMax = 220 * 1024;
    if (bytes <= 48 * 1024) return cudaSuccess;
    if (bytes > kMax) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMax);
}

__device__ __forceinline__ float2 mul_ipow(float2 a, int ell) {
    switch (ell & 3) {
        case 0: return a;
        case 1: return make_float2(-a.y, a.x);
        case 2: return make_float2(-a.x, -a.y);
        default: return make_float2(a.y, -a.x);
    }
}

// Y_lm(k^) / c_lm for integer direction n: Q_l^m(mu) * ((n_x + i n_y)/|n|)^m with
// Q_m^m = 1, Q_{m+1}^m = (2m+1) mu, (l-m) Q_l^m = (2l-1) mu Q_{l-1}^m - (l+m-1) Q_{l-2}^m.
__device__ __forceinline__ float2 ylm_unnorm(int ell, int m, int nx, int ny, int nz, int q) {
    if (q == 0) return make_float2(ell == 0 ? 1.0f : 0.0f, 0.0f);
    const float rinv = rsqrtf((float)q);
    const float mu = (float)nz * rinv;
    float Q;
    if (ell == m) {
        Q = 1.0f;
    } else {
        float q0 = 1.0f, q1 = (float)(2 * m + 1) * mu;
        for (int l = m + 2; l <= ell; ++l) {
            const float q2 = ((float)(2 * l - 1) * mu * q1 - (float)(l + m - 1) * q0) / (float)(l - m);
            q0 = q1;
            q1 = q2;
        }
        Q = q1;
    }
    const float2 rho = make_float2((float)nx * rinv, (float)ny * rinv);
    float2 p = make_float2(Q, 0.0f);
    for (int k = 0; k < m; ++k) p = cmul(p, rho);
    return p;
}

// Z1 ------------------------------------------------------------------------
// Shared radial-table row stride: bins rounded up to 4, plus 4 when that is a
// multiple of 8 (bank skew for the 16-byte reads of a warp).
__host__ __device__ constexpr int zstab_row_stride(int S) {
    return ((S + 3) & ~3) + ((((S + 3) >> 2) & 1) ? 0 : 4);
}

// STAB: the radial factors of the block's columns are first copied into shared
// memory (rows (|n_x|, column), 16-byte asynchronous copies; layout and bank
// skew as the window pass I1), otherwise each element gathers them from the table.
template <int N, bool STAB>
__global__ void __launch_bounds__(ZCfg<N>::TS, 1) k_zeta_x(const float2* __restrict__ spec, float2* __restrict__ fields,
                                                         const HarmBatch hb, const Tables tb) {
    using C = ZCfg<N>;
    constexpr int W = C::W, T = N / 8, H = N / 2;
    extern __shared__ __align__(16) float2 smem[];
    float* ttab = reinterpret_cast<float*>(smem + SmemStrided<W>::words(N));  // [a][col][RS] (STAB)
    const int RS = zstab_row_stride(hb.S);
    const int col = threadIdx.x % W, t = threadIdx.x / W;
    const int ky = blockIdx.y, kz = blockIdx.x * W + col;
    const int ny = signed_freq(ky, N), nz = signed_freq(kz, N);
    const size_t xs = (size_t)N * H;
    const size_t n3 = (size_t)N * N * N;
    if constexpr (STAB) {
        const int S4 = (hb.S + 3) >> 2;
        const int total = H * W * S4;
        for (int e = threadIdx.x; e < total; e += C::TS) {
            const int s4 = e % S4, c = (e / S4) % W, a = e / (S4 * W);
            const int kzc = blockIdx.x * W + c, nzc = signed_freq(kzc, N);
            // Nyquist rows and columns carry K = 0: read row 0, which is always in range
            const int qq = (ky == H || kzc == H) ? 0 : a * a + ny * ny + nzc * nzc;
            const float* src = (hb.tab2 && s4 >= 2) ? hb.tab2 + (size_t)qq * hb.nbp + 4 * (s4 - 2)
                                                     : hb.tab + (size_t)qq * hb.nbp + 4 * s4;
            ac::cp_async16(ttab + (a * W + c) * RS + 4 * s4, src);
        }
        ac::cp_async_commit();
    }
    const float phyz = __ldg(tb.phi + ky) * __ldg(tb.phi + kz);
    float2 v0[8];
    int q[8];  // table index (gather form only)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int kx = t + i * T;
        const int nx = signed_freq(kx, N);
        float2 d;
        if (kz < H) {
            d = spec[(size_t)kx * xs + (size_t)ky * H + kz];
        } else if (kz > H) {  // delta^(n) = conj(delta^(-n)) for a real field
            d = cconj(spec[(size_t)((N - kx) & (N - 1)) * xs + (size_t)((N - ky) & (N - 1)) * H + (N - kz)]);
        } else {
            d = make_float2(0.f, 0.f);
        }
        const bool nyq = (kx == H) || (ky == H) || (kz == H);
        const int qq = nx * nx + ny * ny + nz * nz;
        q[i] = nyq ? 0 : qq;  // table index stays in range on Nyquist lanes
        const float2 y = ylm_unnorm(hb.ell, hb.m, nx, ny, nz, qq);
        const float2 ang = mul_ipow(cscale(y, hb.ylm_norm * __ldg(tb.phi + kx) * phyz), hb.ell);
        v0[i] = nyq ? make_float2(0.f, 0.f) : cmul(d, ang);
    }
    if constexpr (STAB) {
        ac::cp_async_wait_all();
        __syncthreads();
    }
    // Under STAB the row of element i is |n_x| = t + iT (i < 4) or N - t - iT (i >= 4; the
    // Nyquist element t = 0, i = 4 reads row 0): two per-thread bases and constant steps.
    const int qlo = (t * W + col) * RS, qhi = ((N - t) * W + col) * RS;
    auto trow = [&](int i) {
        return i < 4 ? qlo + i * (T * W) * RS : ((t == 0 && i == 4) ? col * RS : qhi - i * (T * W) * RS);
    };
    float2 wc[3 * twiddled_stages<N>()];  // the thread's stage twiddles, the same for every bin
    load_stage_twiddles<N, true>(t, tb.tw, wc);
    const int nbp = hb.nbp;
    const int nf = (hb.S + 1) >> 1;  // packed fields (m = 0)
    for (int g = 0; g < hb.S; g += 4) {
        float4 tv[8];  // radial factors of bins g..g+3: one 16-byte load per element
#pragma unroll
        for (int i = 0; i < 8; ++i)
            tv[i] = STAB ? *reinterpret_cast<const float4*>(ttab + trow(i) + g)
                         : __ldg(reinterpret_cast<const float4*>(
                               (hb.tab2 && g >= 8) ? hb.tab2 + (size_t)q[i] * nbp + (g - 8)
                                                   : hb.tab + (size_t)q[i] * nbp + g));
        if (hb.pack) {  // field f = bins 2f (real part) and 2f + 1 (imaginary part; 0 past the last bin)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int f = (g >> 1) + j;
                if (f >= nf) break;  // uniform across the block
                float2 v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    v[i] = cmul(v0[i], j == 0 ? make_float2(tv[i].x, tv[i].y) : make_float2(tv[i].z, tv[i].w));
                fft_line_wc<N, true>(v, t, tb.tw, SmemStrided<W>{smem, col}, wc);
                float2* dst = fields + (size_t)f * n3 + (size_t)ky * N + kz;
#pragma unroll
                for (int i = 0; i < 8; ++i) dst[(size_t)(t + i * T) * N * N] = v[i];
            }
            continue;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = g + j;
            if (b >= hb.S) break;  // uniform across the block
            float2 v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                v[i] = cscale(v0[i], j == 0 ? tv[i].x : (j == 1 ? tv[i].y : (j == 2 ? tv[i].z : tv[i].w)));
            fft_line_wc<N, true>(v, t, tb.tw, SmemStrided<W>{smem, col}, wc);
            float2* dst = fields + (size_t)b * n3 + (size_t)ky * N + kz;
#pragma unroll
            for (int i = 0; i < 8; ++i) dst[(size_t)(t + i * T) * N * N] = v[i];
        }
    }
}

// Z1 on mirror lines: the x lines at k_y and N - k_y see the same radial factor at every
// element (the same n_y^2), so a block transforms both for its W columns, their FFTs
// exchanging through two tiles behind the same barriers, and one table read serves the two
// lines.  Their angular factors are conjugate: Y_lm(n_x, -n_y, n_z) = conj Y_lm(n_x, n_y, n_z)
// (only the azimuth changes sign), so Y_lm is evaluated once per element.  The radial table
// is staged without padding: the 16-byte chunk j of row r sits at chunk
// j ^ ((r >> rsh) & (RS / 4 - 1)), RS = 4, 8 or 16 floats, so a quarter warp's 16-byte reads
// meet 8 distinct bank groups.  Blocks at k_y = 0 and N/2 (their own mirrors) transform one
// line set.
// PAIRED (8-column tiles): both lines' values of a column go out in one 16-byte store, in
// the paired order of the window pass (16-column groups, line 2 k_y + h of group g holding
// rows k_y and N - k_y of its columns side by side), which the y pass reads
// (k_inv_y_e<..., PAIRED>); grid (N / W, N / 2): the block at k_y = 0 also writes the zero
// k_y = N/2 line.
__host__ __device__ constexpr int zmirror_row_floats(int S) { return S <= 4 ? 4 : (S <= 8 ? 8 : 16); }

template <int N, bool ONE = false, bool PAIRED = false>
__global__ void __launch_bounds__(ZCfg<N>::TS, 1) k_zeta_x_mirror(const float2* __restrict__ spec,
                                                                float2* __restrict__ fields, const HarmBatch hb,
                                                                const Tables tb) {
    using C = ZCfg<N>;
    constexpr int W = C::W, T = N / 8, H = N / 2;
    static_assert(!PAIRED || W == 8, "the paired order pairs two 8-column tiles in a 16-column group");
    constexpr int TILE = SmemStrided<W>::words(N);
    extern __shared__ __align__(16) float2 smem[];
    float* ttab = reinterpret_cast<float*>(smem + 2 * TILE);  // [a][col][RS], chunks swizzled
    const int RS = zmirror_row_floats(hb.S);
    const int rsh = RS == 16 ? 1 : 2, cmask = RS / 4 - 1;
    const int col = threadIdx.x % W, t = threadIdx.x / W;
    const int ky = blockIdx.y, kyb = (N - ky) & (N - 1), kz = blockIdx.x * W + col;  // blockIdx.y in [0, H]
    const bool two = (ky != 0 && ky != H);
    const int ny = signed_freq(ky, N), nz = signed_freq(kz, N);
    const size_t xs = (size_t)N * H;
    const size_t n3 = (size_t)N * N * N;
    {
        const int S4 = (hb.S + 3) >> 2;
        const int total = H * W * S4;
        for (int e = threadIdx.x; e < total; e += C::TS) {
            const int s4 = e % S4, c = (e / S4) % W, a = e / (S4 * W);
            const int kzc = blockIdx.x * W + c, nzc = signed_freq(kzc, N);
            const int qq = (ky == H || kzc == H) ? 0 : a * a + ny * ny + nzc * nzc;
            const float* src = (hb.tab2 && s4 >= 2) ? hb.tab2 + (size_t)qq * hb.nbp + 4 * (s4 - 2)
                                                     : hb.tab + (size_t)qq * hb.nbp + 4 * s4;
            const int row = a * W + c;
            ac::cp_async16(ttab + row * RS + 4 * (s4 ^ ((row >> rsh) & cmask)), src);
        }
        ac::cp_async_commit();
    }
    const float phyz = __ldg(tb.phi + ky) * __ldg(tb.phi + kz);  // Phi^(N - k_y) = Phi^(k_y)
    // delta^ along the x line at (k_y', k_z), with the Hermitian expansion for k_z > N/2
    auto load = [&](int kyl, int kx) {
        if (kz < H) return spec[(size_t)kx * xs + (size_t)kyl * H + kz];
        if (kz > H)
            return cconj(spec[(size_t)((N - kx) & (N - 1)) * xs + (size_t)((N - kyl) & (N - 1)) * H + (N - kz)]);
        return make_float2(0.f, 0.f);
    };
    float2 va0[8], vb0[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int kx = t + i * T;
        const int nx = signed_freq(kx, N);
        const bool nyq = (kx == H) || (ky == H) || (kz == H);
        const int qq = nx * nx + ny * ny + nz * nz;
        const float w = hb.ylm_norm * __ldg(tb.phi + kx) * phyz;
        const float2 y = cscale(ylm_unnorm(hb.ell, hb.m, nx, ny, nz, qq), w);
        va0[i] = nyq ? make_float2(0.f, 0.f) : cmul(load(ky, kx), mul_ipow(y, hb.ell));
        vb0[i] = (nyq || !two) ? make_float2(0.f, 0.f) : cmul(load(kyb, kx), mul_ipow(cconj(y), hb.ell));
    }
    auto trow = [&](int i) {  // |n_x| = t + iT (i < 4) or N - t - iT (the Nyquist element reads row 0)
        const int ax = i < 4 ? t + i * T : ((t == 0 && i == 4) ? 0 : N - t - i * T);
        return ax * W + col;
    };
    ac::cp_async_wait_all();
    __syncthreads();
    float2 wc[3 * twiddled_stages<N>()];
    load_stage_twiddles<N, true>(t, tb.tw, wc);
    const SmemStrided<W> sms[2] = {{smem, col}, {smem + TILE, col}};
    const int nf = (hb.S + 1) >> 1;  // packed fields (m = 0)
    const int nout = hb.pack ? nf : hb.S;
    for (int g = 0; g < hb.S; g += 4) {
        // ONE: each field's factors are read when used instead of four bins' at once
        // (24 registers fewer, so the kernel does not spill)
        float4 tv[ONE ? 1 : 8];
        if constexpr (!ONE) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = trow(i);
                tv[i] = *reinterpret_cast<const float4*>(ttab + r * RS + 4 * ((g >> 2) ^ ((r >> rsh) & cmask)));
            }
        }
        // packed: fields g/2 and g/2 + 1 (bins (2f, 2f + 1) as real and imaginary parts); else bins g..g+3
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int f = hb.pack ? (g >> 1) + j : g + j;
            if ((hb.pack && j >= 2) || f >= nout) break;  // uniform across the block
            float2 v[2][8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if constexpr (ONE) {
                    const int r = trow(i);
                    const float* cp = ttab + r * RS + 4 * ((g >> 2) ^ ((r >> rsh) & cmask));
                    if (hb.pack) {
                        const float2 k2 = *reinterpret_cast<const float2*>(cp + 2 * j);
                        v[0][i] = cmul(va0[i], k2);
                        v[1][i] = cmul(vb0[i], k2);
                    } else {
                        const float k1 = cp[j];
                        v[0][i] = cscale(va0[i], k1);
                        v[1][i] = cscale(vb0[i], k1);
                    }
                } else if (hb.pack) {
                    const float2 k2 = j == 0 ? make_float2(tv[i].x, tv[i].y) : make_float2(tv[i].z, tv[i].w);
                    v[0][i] = cmul(va0[i], k2);
                    v[1][i] = cmul(vb0[i], k2);
                } else {
                    const float k1 = j == 0 ? tv[i].x : (j == 1 ? tv[i].y : (j == 2 ? tv[i].z : tv[i].w));
                    v[0][i] = cscale(va0[i], k1);
                    v[1][i] = cscale(vb0[i], k1);
                }
            }
            fft_lines_wc<N, true, 2>(v, t, sms, wc);
            if constexpr (PAIRED) {
                const int off = t * (N * N) + (2 * ky + (int)(blockIdx.x & 1)) * N + (int)(blockIdx.x >> 1) * 16 + 2 * col;
                float4* dst = reinterpret_cast<float4*>(fields + (size_t)f * n3 + off);
#pragma unroll
                for (int i = 0; i < 8; ++i) {  // (this form of the store spills 8 bytes; a float2 pointer spilled 44)
                    float4 q;
                    q.x = v[0][i].x;
                    q.y = v[0][i].y;
                    q.z = v[1][i].x;
                    q.w = v[1][i].y;
                    dst[(size_t)i * T * N * N / 2] = q;
                }
            } else {
                float2* dst = fields + (size_t)f * n3 + (size_t)kz;
#pragma unroll
                for (int i = 0; i < 8; ++i) dst[(size_t)(t + i * T) * N * N + (size_t)ky * N] = v[0][i];
                if (two) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) dst[(size_t)(t + i * T) * N * N + (size_t)kyb * N] = v[1][i];
                }
            }
        }
    }
}

// Z2: inverse y FFT of every bin field in place (full-length k_z columns, strided tiles):
// launch_zeta_y in fft_passes.cu, whose variants the FFT autotuner picks (pass 3).

// Z3 ------------------------------------------------------------------------
// The 10 tiles (ti, tj), ti <= tj, of a symmetric 16x16 Gram in 4x4 tiles (tile = 4 ti + tj),
// ordered by max(ti, tj): the first 1, 3, 6 or 10 cover the Gram of up to 4, 8, 12 or 16 rows.
__constant__ int kGramTiles[10] = {0, 1, 5, 2, 6, 10, 3, 7, 11, 15};
// Persistent over (x, y) lines.  Per line: GB bin lines per round are inverse
// transformed along z (T threads each) into shared memory; then the 10 upper
// 4x4 bin tiles x 3 z-slices per warp accumulate the Gram, float32 per line, flushed to
// float64 registers every 8 lines.  Partial Gram per block: part[(b1*16+b2)*nblk + blk].
// REAL: the S lines are packed real fields (m = 0): line f holds bins 2f and 2f + 1, and
// the Gram runs over the 2S real components.
template <int N, bool REAL>
__global__ void __launch_bounds__(ZCfg<N>::ZT) k_zeta_z_gram(const float2* __restrict__ fields, int S,
                                                              const float* __restrict__ delta,
                                                              const float2* __restrict__ tw,
                                                              double* __restrict__ part,
                                                              unsigned* __restrict__ err) {
    using C = ZCfg<N>;
    constexpr int T = C::T, GB = C::GB, LPZ = C::LPZ;
    constexpr bool PREF = C::PREFETCH;
    extern __shared__ __align__(16) float2 smem[];
    __shared__ double tot[256];
    __shared__ __align__(8) uint64_t full;
    float* dsm2 = reinterpret_cast<float*>(smem + 16 * LPZ);      // [2][N] delta lines
    float2* stage = reinterpret_cast<float2*>(dsm2 + 2 * N);       // [16][N] bin lines of the next line
    bool late = false;
    const size_t n3 = (size_t)N * N * N;
    const int tid = threadIdx.x;
    const int bb = tid / T, t = tid % T;
    // Gram phase: only the nt tiles that hold Gram rows are computed (nt = 1, 3, 6, 10 for up
    // to 4, 8, 12, 16 rows: S bins, or 2S real parts when REAL).  Lane l < 30 of warp w owns
    // tile kGramTiles[l % nt] and z-slice s = per w + l / nt (per = 30 / nt slices per warp),
    // z = s, s + NS, ... (lanes 30, 31 idle).  With all 10 tiles the 12 addresses a warp reads
    // per z fall on distinct bank pairs.
    const int rows = REAL ? 2 * S : S;
    const int nt = rows <= 4 ? 1 : (rows <= 8 ? 3 : (rows <= 12 ? 6 : 10));
    const int per = 30 / nt;
    const int lane_g = tid & 31, sub = lane_g / nt;
    const bool active = lane_g < 30;
    const int tile = active ? kGramTiles[lane_g % nt] : 0;
    const int ti = tile >> 2, tj = tile & 3;
    const int NS = (int)(blockDim.x >> 5) * per;
    const int zs = (tid >> 5) * per + sub;
    float acc[4][4];
    double acc64[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            acc[a][b] = 0.0f;
            acc64[a][b] = 0.0;
        }
    const int rounds = (S + GB - 1) / GB;
    int since_flush = 0;
    float2 wc[3 * twiddled_stages<N>()];  // the thread's stage twiddles, the same for every bin line
    load_stage_twiddles<N, true>(t, tw, wc);
    // fetch the S bin lines and the delta line of `line` by bulk copies
    auto fetch = [&](size_t ln, int slot) {
        ac::mbar_expect_tx(&full, (uint32_t)(S * N * sizeof(float2) + N * sizeof(float)));
        for (int b = 0; b < S; ++b) ac::bulk_g2s(stage + b * N, fields + (size_t)b * n3 + ln * N, N * sizeof(float2), &full);
        ac::bulk_g2s(dsm2 + slot * N, delta + ln * N, N * sizeof(float), &full);
    };
    if constexpr (PREF) {
        if (tid == 0) {
            ac::mbar_init(&full, 1);
            ac::mbar_init_fence();
        }
        __syncthreads();
        if (tid == 0 && blockIdx.x < (size_t)N * N) fetch(blockIdx.x, 0);
    }
    int it = 0;
    for (size_t line = blockIdx.x; line < (size_t)N * N; line += gridDim.x, ++it) {
        if constexpr (PREF) {
            if (!ac::mbar_wait(&full, it & 1)) late = true;
        }
        for (int r = 0; r < rounds; ++r) {
            const int b = r * GB + bb;
            // lines past the last bin hold no data; where a line owns whole warps (N >= 256)
            // they skip the transform (their Gram products are never read)
            if (T >= 32 && b >= S) continue;
            float2 v[8];
            if (b < S) {
                if constexpr (PREF) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] = stage[b * N + t + i * T];
                } else {
                    const float2* src = fields + (size_t)b * n3 + line * N;
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] = src[t + i * T];
                }
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = make_float2(0.f, 0.f);
            }
            const SmemZLine<N> sm{{smem + b * LPZ}, bb};  // threads of group bb only
            fft_line_wc<N, true>(v, t, tw, sm, wc);
#pragma unroll
            for (int i = 0; i < 8; ++i) sm.st(t + i * T, v[i]);
        }
        float* dsm = dsm2 + (PREF ? (it & 1) * N : 0);
        if constexpr (!PREF) {
            for (int z = tid; z < N; z += blockDim.x) dsm[z] = delta[line * N + z];
        }
        __syncthreads();  // the stage has been read: fetch the next line during the Gram phase
        if constexpr (PREF) {
            if (tid == 0 && line + gridDim.x < (size_t)N * N) {
                ac::fence_proxy_async();
                fetch(line + gridDim.x, (it + 1) & 1);
            }
        }
        if (REAL && active) {
            for (int z = zs; z < N; z += NS) {
                const float d = dsm[z];
                const int zp = SmemLine<N>::at(z);
                // rows 4 ti .. 4 ti + 3 are lines 2 ti, 2 ti + 1 (real, imaginary parts)
                const float2 p0 = smem[(2 * ti) * LPZ + zp], p1 = smem[(2 * ti + 1) * LPZ + zp];
                const float2 r0 = smem[(2 * tj) * LPZ + zp], r1 = smem[(2 * tj + 1) * LPZ + zp];
                const float x[4] = {p0.x * d, p0.y * d, p1.x * d, p1.y * d};
                const float y[4] = {r0.x, r0.y, r1.x, r1.y};
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int k2 = 0; k2 < 4; ++k2) acc[k][k2] = fmaf(x[k], y[k2], acc[k][k2]);
            }
        } else if (active) {
            for (int z = zs; z < N; z += NS) {
                const float d = dsm[z];
                const int zp = SmemLine<N>::at(z);
                float2 a1[4], a2[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    a1[k] = smem[(4 * ti + k) * LPZ + zp];
                    a2[k] = smem[(4 * tj + k) * LPZ + zp];
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 e = cscale(a1[k], d);
#pragma unroll
                    for (int k2 = 0; k2 < 4; ++k2) acc[k][k2] = fmaf(e.x, a2[k2].x, fmaf(e.y, a2[k2].y, acc[k][k2]));
                }
            }
        }
        if (++since_flush == 8) {
            since_flush = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc64[a][b] += (double)acc[a][b];
                    acc[a][b] = 0.0f;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc64[a][b] += (double)acc[a][b];
    // lanes l, l + nt, l + 2 nt, ... < 30 hold the same tile: merge onto lane l, then warps
    // add in turn
    for (int k = 1; k < per; ++k) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const double v = __shfl_down_sync(0xffffffffu, acc64[a][b], k * nt);
                if (lane_g < nt) acc64[a][b] += v;
            }
    }
    for (int e = tid; e < 256; e += blockDim.x) tot[e] = 0.0;
    __syncthreads();
    const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) {
        if (wid == w && lane < nt) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) tot[(4 * ti + a) * 16 + (4 * tj + b)] += acc64[a][b];
        }
        __syncthreads();
    }
    for (int e = tid; e < 256; e += blockDim.x) part[(size_t)e * gridDim.x + blockIdx.x] = tot[e];
    if (late && (tid & 31) == 0) atomicOr(err, 4u);
}

// Z3, two blocks per SM (N = 512): the same transforms and Gram as k_zeta_z_gram in half
// the resources, so that two blocks share each SM and one block's transforms overlap the
// other's Gram phase instead of every warp of the SM waiting on the same barriers.  Bin
// lines are loaded straight into registers (no bulk-copy stage), the float32 Gram tile of
// each lane is flushed every 8 lines into float64 tiles per warp in shared memory, and the
// kernel is held to 64 registers.
template <int N>
struct Z2Cfg {
    static constexpr int T = N / 8;          // threads per bin line
    static constexpr int GB = 512 / T;       // bin lines per round
    static constexpr int THREADS = GB * T;   // 512
    static constexpr int NW = THREADS / 32;
    static constexpr int LPZ = ZCfg<N>::LPZ;
    static constexpr size_t SMEM = (size_t)16 * LPZ * sizeof(float2)    // transformed bin lines
                                   + (size_t)N * sizeof(float)          // delta line
                                   + (size_t)NW * 160 * sizeof(double);  // float64 tiles per warp
};

template <int N, bool REAL>
__global__ void __launch_bounds__(Z2Cfg<N>::THREADS, 2) k_zeta_z_gram2(const float2* __restrict__ fields, int S,
                                                                      const float* __restrict__ delta,
                                                                      const float2* __restrict__ tw,
                                                                      double* __restrict__ part) {
    using C = Z2Cfg<N>;
    constexpr int T = C::T, GB = C::GB, LPZ = C::LPZ, NW = C::NW;
    extern __shared__ __align__(16) float2 smem[];
    float* dsm = reinterpret_cast<float*>(smem + 16 * LPZ);          // [N]
    double* wacc = reinterpret_cast<double*>(dsm + N);               // [NW][10][16]
    const size_t n3 = (size_t)N * N * N;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int bb = tid / T, t = tid % T;
    // Gram lanes as in k_zeta_z_gram: nt tiles that hold rows, 30 lanes per warp spread over them
    const int rows = REAL ? 2 * S : S;
    const int nt = rows <= 4 ? 1 : (rows <= 8 ? 3 : (rows <= 12 ? 6 : 10));
    const int per = 30 / nt;
    const int sub = lane / nt;
    const bool active = lane < 30;
    const int tile = active ? kGramTiles[lane % nt] : 0;
    const int ti = tile >> 2, tj = tile & 3;
    const int NS = NW * per;
    const int zs = wid * per + sub;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.0f;
    for (int e = tid; e < NW * 160; e += C::THREADS) wacc[e] = 0.0;
    // the sum of the lanes that hold the same tile goes into the warp's float64 tile
    auto flush = [&]() {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float v = acc[a][c];
                for (int k = 1; k < per; ++k) v += __shfl_down_sync(0xffffffffu, acc[a][c], k * nt);
                if (lane < nt) wacc[(wid * 10 + lane) * 16 + a * 4 + c] += (double)v;
                acc[a][c] = 0.0f;
            }
    };
    const int rounds = (S + GB - 1) / GB;
    int since_flush = 0;
    __syncthreads();
    for (size_t line = blockIdx.x; line < (size_t)N * N; line += gridDim.x) {
        for (int r = 0; r < rounds; ++r) {
            const int b = r * GB + bb;
            if (T >= 32 && b >= S) continue;  // no data; the whole line group skips
            float2 v[8];
            if (b < S) {
                const float2* src = fields + (size_t)b * n3 + line * N;
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = src[t + i * T];
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = make_float2(0.f, 0.f);
            }
            const SmemZLine<N> sm{{smem + b * LPZ}, bb};
            fft_line<N, true>(v, t, tw, sm);
#pragma unroll
            for (int i = 0; i < 8; ++i) sm.st(t + i * T, v[i]);
        }
        for (int z = tid; z < N; z += C::THREADS) dsm[z] = delta[line * N + z];
        __syncthreads();
        if (REAL && active) {
            for (int z = zs; z < N; z += NS) {
                const float d = dsm[z];
                const int zp = SmemLine<N>::at(z);
                const float2 p0 = smem[(2 * ti) * LPZ + zp], p1 = smem[(2 * ti + 1) * LPZ + zp];
                const float2 r0 = smem[(2 * tj) * LPZ + zp], r1 = smem[(2 * tj + 1) * LPZ + zp];
                const float x[4] = {p0.x * d, p0.y * d, p1.x * d, p1.y * d};
                const float y[4] = {r0.x, r0.y, r1.x, r1.y};
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int k2 = 0; k2 < 4; ++k2) acc[k][k2] = fmaf(x[k], y[k2], acc[k][k2]);
            }
        } else if (active) {
            for (int z = zs; z < N; z += NS) {
                const float d = dsm[z];
                const int zp = SmemLine<N>::at(z);
                float2 a1[4], a2[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    a1[k] = smem[(4 * ti + k) * LPZ + zp];
                    a2[k] = smem[(4 * tj + k) * LPZ + zp];
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 e = cscale(a1[k], d);
#pragma unroll
                    for (int k2 = 0; k2 < 4; ++k2) acc[k][k2] = fmaf(e.x, a2[k2].x, fmaf(e.y, a2[k2].y, acc[k][k2]));
                }
            }
        }
        if (++since_flush == 8) {
            since_flush = 0;
            flush();
        }
        __syncthreads();
    }
    flush();
    __syncthreads();
    // entry (b1, b2) of the upper triangle by tiles: the sum over warps of the float64 tiles
    for (int e = tid; e < 256; e += C::THREADS) {
        const int b1 = e >> 4, b2 = e & 15, gi = b1 >> 2, gj = b2 >> 2;
        double s = 0.0;
        if (gi <= gj) {
            const int code = 4 * gi + gj;
            int idx = 0;
            while (idx < 10 && kGramTiles[idx] != code) ++idx;
            if (idx < nt) {
                const int slot = idx * 16 + (b1 & 3) * 4 + (b2 & 3);
                for (int w = 0; w < NW; ++w) s += wacc[w * 160 + slot];
            }
        }
        part[(size_t)e * gridDim.x + blockIdx.x] = s;
    }
}

// Z3 on the tensor cores ---------------------------------------------------
// Same line loop and z transforms as k_zeta_z_gram; the Gram runs on tcgen05.
// With K = (z, Re/Im) the Gram is a plain product G = A B:
//   A[r][k] = delta(z) * X_b(k),  B[k][c] = X_b'(k),  X_b(2z) = Re a_b(z), X_b(2z+1) = Im a_b(z).
// Split precision with TF32: x = x_hi + x_lo (x_hi = tf32(x), x_lo = x - x_hi),
// one MMA computes every needed term: A rows = [Y_hi (16 bins); Y_lo (16 bins);
// 96 zero rows] (M = 128), B columns = [X_hi | X_lo] (N = 32), so
//   G = D[0:16, 0:16] + D[0:16, 16:32] + D[16:32, 0:16]   (hi*hi + hi*lo + lo*hi)
// with D accumulated in float32 in tensor memory over one line and drained to
// float64 (two accumulators alternate between lines).  Operands are staged in shared memory in the no-swizzle K-major
// layout (8-row x 16-byte core matrices), K chunks of 64, double-buffered; one
// thread issues the MMAs and commits them to an mbarrier per buffer.  Every
// wait is bounded: on expiry the kernel sets err bit 2 and carries on, so the
// host reports HERMES_ERR_TIMEOUT instead of hanging.
namespace tc {
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the completion of phase `parity` of barrier b; false after one second.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) { return ac::mbar_wait(b, parity); }
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
// shared-memory matrix descriptor: no swizzle, K-major, start / LBO / SBO in bytes
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// kind::tf32, D f32, A and B K-major, M = 128, N = 32
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
constexpr int KCH = 64;                 // K elements per staged chunk (32 z values)
constexpr int CORE_ROW_GROUP = 2048;    // bytes between 8-row groups (16 K core matrices x 128 B)
constexpr int A_BYTES = 128 * KCH * 4;  // 32 KiB
constexpr int B_BYTES = 32 * KCH * 4;   // 8 KiB
__device__ __forceinline__ uint32_t off(int r, int k) {
    return (uint32_t)((r >> 3) * CORE_ROW_GROUP + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}
}  // namespace tc

template <int N>
struct ZTcCfg {
    static constexpr int LPZ = ZCfg<N>::LPZ;
    static constexpr size_t OPS = 2 * (size_t)(tc::A_BYTES + tc::B_BYTES);  // 80 KiB, 1024-aligned start
    static constexpr size_t SMEM = OPS + (size_t)16 * LPZ * sizeof(float2) + (size_t)N * sizeof(float);
};

template <int N>
__global__ void __launch_bounds__(ZCfg<N>::ZT, 1) k_zeta_z_gram_tc(const float2* __restrict__ fields, int S,
                                                                    const float* __restrict__ delta,
                                                                    const float2* __restrict__ tw,
                                                                    double* __restrict__ part,
                                                                    unsigned* __restrict__ err) {
    using C = ZCfg<N>;
    constexpr int T = C::T, GB = C::GB, LPZ = C::LPZ;
    extern __shared__ __align__(1024) unsigned char zsm[];
    unsigned char* opA = zsm;                                   // 2 x A chunk
    unsigned char* opB = zsm + 2 * tc::A_BYTES;                 // 2 x B chunk
    float2* E = reinterpret_cast<float2*>(zsm + ZTcCfg<N>::OPS);  // 16 transformed bin lines
    float* dsm = reinterpret_cast<float*>(E + 16 * LPZ);
    __shared__ __align__(8) uint64_t mbar[2];   // "empty": MMAs reading buffer b finished
    __shared__ __align__(8) uint64_t fullb[2];  // "full": every warp wrote its part of buffer b
    __shared__ uint32_t tmem_slot;
    const size_t n3 = (size_t)N * N * N;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int bb = tid / T, t = tid % T;

    // zero the operand buffers once (rows 32..127 of A stay zero for good)
    for (int e = tid; e < (int)(ZTcCfg<N>::OPS / 16); e += blockDim.x)
        reinterpret_cast<float4*>(zsm)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    constexpr int NWARPS = ZCfg<N>::ZT / 32;
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_init(&fullb[0], NWARPS);
        tc::mbar_init(&fullb[1], NWARPS);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (wid == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(tc::su32(&tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t dtm = tmem_slot;

    double acc64[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc64[c] = 0.0;
    uint32_t uses[2] = {0, 0}, done[2] = {0, 0};
    bool timed_out = false;
    const int rounds = (S + GB - 1) / GB;

    // Line L accumulates into TMEM columns [32 (L & 1), +32).  The accumulator of
    // line L-1 is drained to float64 while line L is transformed, so each float32
    // accumulation runs over one line (K = 2N) only.
    auto wait_all = [&]() {
#pragma unroll
        for (int bf = 0; bf < 2; ++bf)
            if (done[bf] < uses[bf]) {
                if (!tc::mbar_wait(&mbar[bf], (uses[bf] - 1) & 1)) timed_out = true;
                done[bf] = uses[bf];
            }
    };
    auto drain = [&](uint32_t col) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (wid == 0) {
            uint32_t r[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(dtm + col));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            // row = lane: rows 0..15 hold hi*hi (cols 0..15) and hi*lo (16..31); rows 16..31 lo*hi
#pragma unroll
            for (int c = 0; c < 16; ++c)
                acc64[c] += (double)__uint_as_float(r[c]) + (lane < 16 ? (double)__uint_as_float(r[16 + c]) : 0.0);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    };

    int nlines = 0;
    for (size_t line = blockIdx.x; line < (size_t)N * N; line += gridDim.x, ++nlines) {
        for (int r = 0; r < rounds; ++r) {
            const int b = r * GB + bb;
            float2 v[8];
            if (b < S) {
                const float2* src = fields + (size_t)b * n3 + line * N;
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = src[t + i * T];
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = make_float2(0.f, 0.f);
            }
            const SmemLine<N> sm{E + b * LPZ};
            fft_line<N, true>(v, t, tw, sm);
#pragma unroll
            for (int i = 0; i < 8; ++i) sm.st(t + i * T, v[i]);
        }
        for (int z = tid; z < N; z += blockDim.x) dsm[z] = delta[line * N + z];
        if (nlines > 0) {  // line L-1 is complete by now in all likelihood: drain its accumulator
            wait_all();
            drain(32u * (uint32_t)((nlines - 1) & 1));
        }
        __syncthreads();
        const uint32_t dcol = dtm + 32u * (uint32_t)(nlines & 1);
        for (int z0 = 0; z0 < N; z0 += tc::KCH / 2) {
            const int bf = (int)((uses[0] + uses[1]) & 1);
            if (done[bf] < uses[bf]) {  // the MMAs that last read this buffer must be finished
                if (!tc::mbar_wait(&mbar[bf], (uses[bf] - 1) & 1)) timed_out = true;
                done[bf] = uses[bf];
            }
            unsigned char* A = opA + bf * tc::A_BYTES;
            unsigned char* B = opB + bf * tc::B_BYTES;
            for (int e = tid; e < 16 * (tc::KCH / 2); e += blockDim.x) {
                const int b = e & 15, zl = e >> 4, z = z0 + zl;
                const float2 x = E[b * LPZ + SmemLine<N>::at(z)];
                const float d = dsm[z];
                const float yr = d * x.x, yi = d * x.y;
                const uint32_t xrh = tc::to_tf32(x.x), xih = tc::to_tf32(x.y);
                const uint32_t yrh = tc::to_tf32(yr), yih = tc::to_tf32(yi);
                const float xrl = x.x - __uint_as_float(xrh), xil = x.y - __uint_as_float(xih);
                const float yrl = yr - __uint_as_float(yrh), yil = yi - __uint_as_float(yih);
                const int k = 2 * zl;
                *reinterpret_cast<float2*>(A + tc::off(b, k)) = make_float2(__uint_as_float(yrh), __uint_as_float(yih));
                *reinterpret_cast<float2*>(A + tc::off(16 + b, k)) = make_float2(yrl, yil);
                *reinterpret_cast<float2*>(B + tc::off(b, k)) = make_float2(__uint_as_float(xrh), __uint_as_float(xih));
                *reinterpret_cast<float2*>(B + tc::off(16 + b, k)) = make_float2(xrl, xil);
            }
            // make this thread's operand stores visible to the tensor-core proxy, then
            // one arrival per warp on the buffer's "full" barrier
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::su32(&fullb[bf])) : "memory");
            if (tid == 0) {
                if (!tc::mbar_wait(&fullb[bf], uses[bf] & 1)) timed_out = true;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = tc::su32(A), b0 = tc::su32(B);
#pragma unroll
                for (int kk = 0; kk < tc::KCH / 8; ++kk) {
                    const uint64_t ad = tc::desc(a0 + kk * 256, 128, tc::CORE_ROW_GROUP);
                    const uint64_t bd = tc::desc(b0 + kk * 256, 128, tc::CORE_ROW_GROUP);
                    const uint32_t accum = (z0 == 0 && kk == 0) ? 0u : 1u;  // each line starts afresh
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dcol),
                        "l"(ad), "l"(bd), "r"(tc::IDESC), "r"(accum));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 tc::su32(&mbar[bf]))
                             : "memory");
            }
            __syncwarp();
            ++uses[bf];
        }
    }
    wait_all();
    if (nlines > 0) drain(32u * (uint32_t)((nlines - 1) & 1));
    __syncthreads();
    if (timed_out && lane == 0) atomicOr(err, 2u);
    // rows 0..15 plus rows 16..31 (lo*hi): G[row][c]
#pragma unroll
    for (int c = 0; c < 16; ++c) acc64[c] += __shfl_down_sync(0xffffffffu, acc64[c], 16);
    if (wid == 0 && lane < 16) {
#pragma unroll
        for (int c = 0; c < 16; ++c) part[(size_t)(lane * 16 + c) * gridDim.x + blockIdx.x] = acc64[c];
    }
    __syncthreads();
    if (wid == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(dtm));
}

// The tensor-core Gram runs for N >= 32 when HERMES_ZETA_TC=1.  It is correct
// (split-TF32, parity-tested) but not the default: the pass is bound by loading
// the bin lines and by the z transforms' block barriers (tensor pipe ~5% busy),
// and the per-chunk operand staging makes it slower than the SIMT Gram.
static bool zeta_tc_enabled(int N) {
    if (N < 32) return false;
    const char* env = getenv("HERMES_ZETA_TC");
    return env && env[0] == '1';
}

template <int N>
static int zeta_blocks_impl() {
    const int lines = N * N;
    const int cap = zeta_tc_enabled(N) ? 148 : 296;  // the tensor-core kernel keeps one CTA per SM
    return lines < cap ? lines : cap;
}

int zeta_z_blocks(int N) {
    switch (N) {
        case 16: return zeta_blocks_impl<16>();
        case 32: return zeta_blocks_impl<32>();
        case 64: return zeta_blocks_impl<64>();
        case 128: return zeta_blocks_impl<128>();
        case 256: return zeta_blocks_impl<256>();
        case 512: return zeta_blocks_impl<512>();
        case 1024: return zeta_blocks_impl<1024>();
    }
    return 0;
}

// The x pass of one (l, m) batch: variant 0 one line set at a time (shared table when it
// fits, gathered factors otherwise), variant 1 the mirror lines together (256^3 and 512^3,
// when the unpadded table and two tiles fit), 2 the same reading each field's factors when
// used, 3 (512^3) the same in the paired order (it never falls back to another form: the
// y pass that follows reads that order).
struct ZetaXArgs {
    const float2* spec;
    float2* fields;
    const HarmBatch* hb;
    const Tables* tb;
    bool use_stab;
    size_t stab_bytes;
    cudaStream_t st;
};
template <int N>
static cudaError_t launch_zeta_x(int var, const ZetaXArgs& a) {
    using C = ZCfg<N>;
    cudaError_t e;
    if constexpr (N == 256 || N == 512) {
        const size_t bytes = 2 * C::SMEM_X + (size_t)(N / 2) * C::W * zmirror_row_floats(a.hb->S) * sizeof(float);
        if (var == 1 && bytes <= 220 * 1024) {
            if ((e = allow_smem_z(k_zeta_x_mirror<N, false>, bytes)) != cudaSuccess) return e;
            k_zeta_x_mirror<N, false><<<dim3(N / C::W, N / 2 + 1, 1), C::TS, bytes, a.st>>>(a.spec, a.fields, *a.hb,
                                                                                           *a.tb);
            return cudaGetLastError();
        }
        if (var == 2 && bytes <= 220 * 1024) {
            if ((e = allow_smem_z(k_zeta_x_mirror<N, true>, bytes)) != cudaSuccess) return e;
            k_zeta_x_mirror<N, true><<<dim3(N / C::W, N / 2 + 1, 1), C::TS, bytes, a.st>>>(a.spec, a.fields, *a.hb,
                                                                                          *a.tb);
            return cudaGetLastError();
        }
        if constexpr (N == 512) {
            if (var == 3) {
                if (bytes > 220 * 1024) return cudaErrorInvalidValue;
                if ((e = allow_smem_z(k_zeta_x_mirror<N, true, true>, bytes)) != cudaSuccess) return e;
                k_zeta_x_mirror<N, true, true><<<dim3(N / C::W, N / 2, 1), C::TS, bytes, a.st>>>(a.spec, a.fields,
                                                                                               *a.hb, *a.tb);
                return cudaGetLastError();
            }
        }
    }
    const dim3 g1(N / C::W, N, 1);
    if (a.use_stab) k_zeta_x<N, true><<<g1, C::TS, a.stab_bytes, a.st>>>(a.spec, a.fields, *a.hb, *a.tb);
    else k_zeta_x<N, false><<<g1, C::TS, C::SMEM_X, a.st>>>(a.spec, a.fields, *a.hb, *a.tb);
    return cudaGetLastError();
}
template <int N>
static cudaError_t zeta_x_trial(int v, void* arg) {
    return launch_zeta_x<N>(v, *static_cast<const ZetaXArgs*>(arg));
}

template <int N>
static cudaError_t zeta_impl(const float2* spec, float2* fields, const float* delta, const HarmBatch& hb,
                             const Tables& tb, double* gram_part, unsigned* err, cudaStream_t st, const Tracer& tr) {
    using C = ZCfg<N>;
    cudaError_t e;
    const size_t stab_bytes = C::SMEM_X + (size_t)(N / 2) * C::W * zstab_row_stride(hb.S) * sizeof(float);
    const bool use_stab = stab_bytes <= 220 * 1024;
    if ((e = allow_smem_z(k_zeta_x<N, false>, C::SMEM_X)) != cudaSuccess) return e;
    if (use_stab && (e = allow_smem_z(k_zeta_x<N, true>, stab_bytes)) != cudaSuccess) return e;
    // m = 0: real fields, two bins per transform (the opt-in tensor-core Gram takes them unpacked)
    HarmBatch hp = hb;
    hp.pack = (hb.m == 0 && hb.S > 1 && !zeta_tc_enabled(N)) ? 1 : 0;
    const int nf = hp.pack ? (hb.S + 1) / 2 : hb.S;  // complex fields transformed
    // the y-pass variant (tuned on the first field before the x pass writes the fields)
    const int yvar = zeta_y_variant(N, fields, nf, tb.tw, st);
    // the x-pass variant, tuned per packing on the first zeta call that uses it (its trials
    // write the fields, which the real launch overwrites)
    const ZetaXArgs xa{spec, fields, &hp, &tb, use_stab, stab_bytes, st};
    const int xv = tuned_variant(N, hp.pack ? 5 : 4, st, zeta_x_trial<N>, const_cast<ZetaXArgs*>(&xa));
    // the paired order of the x pass needs a y pass that reads it; otherwise the same x
    // pass runs with plain stores
    const size_t mbytes = 2 * C::SMEM_X + (size_t)(N / 2) * C::W * zmirror_row_floats(hp.S) * sizeof(float);
    const bool paired = N == 512 && xv == 3 && mbytes <= 220 * 1024 && zeta_y_reads_paired(N, yvar);
    const int xrun = (N == 512 && xv == 3 && !paired) ? 2 : xv;
    tr(K_ZETA_X, 0, st);
    if ((e = launch_zeta_x<N>(xrun, xa)) != cudaSuccess) return e;
    tr(K_ZETA_X, 1, st);
    tr(K_ZETA_Y, 0, st);
    if ((e = launch_zeta_y(N, yvar, fields, nf, tb.tw, st, paired)) != cudaSuccess) return e;
    tr(K_ZETA_Y, 1, st);
    if constexpr (N >= 32) {
        if (zeta_tc_enabled(N)) {
            if ((e = allow_smem_z(k_zeta_z_gram_tc<N>, ZTcCfg<N>::SMEM)) != cudaSuccess) return e;
            tr(K_ZETA_Z_GRAM_TC, 0, st);
            k_zeta_z_gram_tc<N><<<zeta_blocks_impl<N>(), C::ZT, ZTcCfg<N>::SMEM, st>>>(fields, hb.S, delta, tb.tw,
                                                                                    gram_part, err);
            tr(K_ZETA_Z_GRAM_TC, 1, st);
            return cudaGetLastError();
        }
    }
    tr(K_ZETA_Z_GRAM, 0, st);
    if constexpr (N == 256 || N == 512) {
        // two blocks per SM (the bench's zeta step: 219 ms in this pass against 227 for one block)
        const int nblk = zeta_blocks_impl<N>();
        if (hp.pack) {
            if ((e = allow_smem_z(k_zeta_z_gram2<N, true>, Z2Cfg<N>::SMEM)) != cudaSuccess) return e;
            k_zeta_z_gram2<N, true><<<nblk, Z2Cfg<N>::THREADS, Z2Cfg<N>::SMEM, st>>>(fields, nf, delta, tb.tw,
                                                                                  gram_part);
        } else {
            if ((e = allow_smem_z(k_zeta_z_gram2<N, false>, Z2Cfg<N>::SMEM)) != cudaSuccess) return e;
            k_zeta_z_gram2<N, false><<<nblk, Z2Cfg<N>::THREADS, Z2Cfg<N>::SMEM, st>>>(fields, hb.S, delta, tb.tw,
                                                                                   gram_part);
        }
    } else {
        if (hp.pack) {
            if ((e = allow_smem_z(k_zeta_z_gram<N, true>, C::SMEM_Z)) != cudaSuccess) return e;
            k_zeta_z_gram<N, true><<<zeta_blocks_impl<N>(), C::ZT, C::SMEM_Z, st>>>(fields, nf, delta, tb.tw,
                                                                                   gram_part, err);
        } else {
            if ((e = allow_smem_z(k_zeta_z_gram<N, false>, C::SMEM_Z)) != cudaSuccess) return e;
            k_zeta_z_gram<N, false><<<zeta_blocks_impl<N>(), C::ZT, C::SMEM_Z, st>>>(fields, hb.S, delta, tb.tw,
                                                                                    gram_part, err);
        }
    }
    tr(K_ZETA_Z_GRAM, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_zeta_lm(int N, const float2* spec, float2* fields, const float* delta, const HarmBatch& hb,
                           const Tables& tb, double* gram_part, unsigned* err, cudaStream_t st, const Tracer& tr) {
    if (hb.S < 1 || hb.S > 16) return cudaErrorInvalidValue;
    switch (N) {
        case 16: return zeta_impl<16>(spec, fields, delta, hb, tb, gram_part, err, st, tr);
        case 32: return zeta_impl<32>(spec, fields, delta, hb, tb, gram_part, err, st, tr);
        case 64: return zeta_impl<64>(spec, fields, delta, hb, tb, gram_part, err, st, tr);
        case 128: return zeta_impl<128>(spec, fields, delta, hb, tb, gram_part, err, st, tr);
        case 256: return zeta_impl<256>(spec, fields, delta, hb, tb, gram_part, err, st, tr);
        case 512: return zeta_impl<512>(spec, fields, delta, hb, tb, gram_part, err, st, tr);
        case 1024: return zeta_impl<1024>(spec, fields, delta, hb, tb, gram_part, err, st, tr);
    }
    return cudaErrorInvalidValue;
}

}  // namespace hermes
