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
// negative m recovered by conjugation as in Sec. 4.4).
#include "kernels.h"
#include "fft_core.cuh"

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
    static constexpr size_t SMEM_Z = (size_t)16 * LPZ * sizeof(float2) + (size_t)N * sizeof(float);
};
static_assert(ZCfg<16>::ZPER >= 1 && ZCfg<1024>::NZS == 32, "z-pass layout");

template <class K>
static cudaError_t allow_smem_z(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
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
template <int N>
__global__ void __launch_bounds__(ZCfg<N>::TS, 1) k_zeta_x(const float2* __restrict__ spec, float2* __restrict__ fields,
                                                         const HarmBatch hb, const Tables tb) {
    using C = ZCfg<N>;
    constexpr int W = C::W, T = N / 8, H = N / 2;
    extern __shared__ float2 smem[];
    const int col = threadIdx.x % W, t = threadIdx.x / W;
    const int ky = blockIdx.y, kz = blockIdx.x * W + col;
    const int ny = signed_freq(ky, N), nz = signed_freq(kz, N);
    const size_t xs = (size_t)N * H;
    const size_t n3 = (size_t)N * N * N;
    const float phyz = __ldg(tb.phi + ky) * __ldg(tb.phi + kz);
    float2 v0[8];
    int q[8];
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
    const int nbp = hb.nbp;
    for (int g = 0; g < hb.S; g += 4) {
        float4 tv[8];  // radial factors of bins g..g+3: one 16-byte load per element
#pragma unroll
        for (int i = 0; i < 8; ++i) tv[i] = __ldg(reinterpret_cast<const float4*>(hb.tab + (size_t)q[i] * nbp + g));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int b = g + j;
            if (b >= hb.S) break;  // uniform across the block
            float2 v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                v[i] = cscale(v0[i], j == 0 ? tv[i].x : (j == 1 ? tv[i].y : (j == 2 ? tv[i].z : tv[i].w)));
            fft_line<N, true>(v, t, tb.tw, SmemStrided<W>{smem, col});
            float2* dst = fields + (size_t)b * n3 + (size_t)ky * N + kz;
#pragma unroll
            for (int i = 0; i < 8; ++i) dst[(size_t)(t + i * T) * N * N] = v[i];
        }
    }
}

// Z2 is k_strided<N, true> from fft_passes.cu instantiated here for full-length k_z.
template <int N>
__global__ void __launch_bounds__(ZCfg<N>::TS) k_zeta_y(float2* __restrict__ fields, const float2* __restrict__ tw) {
    using C = ZCfg<N>;
    constexpr int W = C::W, T = N / 8;
    extern __shared__ float2 smem[];
    const int col = threadIdx.x % W, t = threadIdx.x / W;
    // block (kz chunk, x, bin); element (y) at stride N
    float2* base = fields + (size_t)blockIdx.z * N * N * N + (size_t)blockIdx.y * N * N + (size_t)blockIdx.x * W + col;
    float2 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = base[(size_t)(t + i * T) * N];
    fft_line<N, true>(v, t, tw, SmemStrided<W>{smem, col});
#pragma unroll
    for (int i = 0; i < 8; ++i) base[(size_t)(t + i * T) * N] = v[i];
}

// Z3 ------------------------------------------------------------------------
// Persistent over (x, y) lines.  Per line: GB bin lines per round are inverse
// transformed along z (T threads each) into shared memory; then 16 tiles of
// 4x4 bins x NZS z-slices accumulate the Gram, float32 per line, flushed to
// float64 registers every 8 lines.  Partial Gram per block: part[(b1*16+b2)*nblk + blk].
template <int N>
__global__ void __launch_bounds__(ZCfg<N>::ZT) k_zeta_z_gram(const float2* __restrict__ fields, int S,
                                                              const float* __restrict__ delta,
                                                              const float2* __restrict__ tw,
                                                              double* __restrict__ part) {
    using C = ZCfg<N>;
    constexpr int T = C::T, GB = C::GB, LPZ = C::LPZ, ZPER = C::ZPER;
    extern __shared__ float2 smem[];
    __shared__ double tot[256];
    float* dsm = reinterpret_cast<float*>(smem + 16 * LPZ);
    const size_t n3 = (size_t)N * N * N;
    const int tid = threadIdx.x;
    const int bb = tid / T, t = tid % T;
    const int tile = tid & 15, zs = tid >> 4;
    const int ti = tile >> 2, tj = tile & 3;
    const bool active = ti <= tj;
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
    for (size_t line = blockIdx.x; line < (size_t)N * N; line += gridDim.x) {
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
            const SmemLine<N> sm{smem + b * LPZ};
            fft_line<N, true>(v, t, tw, sm);
#pragma unroll
            for (int i = 0; i < 8; ++i) sm.st(t + i * T, v[i]);
        }
        for (int z = tid; z < N; z += blockDim.x) dsm[z] = delta[line * N + z];
        __syncthreads();
        if (active) {
            const int z0 = zs * ZPER;
            for (int z = z0; z < z0 + ZPER; ++z) {
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
    // lanes l and l^16 hold the same tile: merge, then warps add in turn
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc64[a][b] += __shfl_xor_sync(0xffffffffu, acc64[a][b], 16);
    for (int e = tid; e < 256; e += blockDim.x) tot[e] = 0.0;
    __syncthreads();
    const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) {
        if (wid == w && lane < 16 && active) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) tot[(4 * ti + a) * 16 + (4 * tj + b)] += acc64[a][b];
        }
        __syncthreads();
    }
    for (int e = tid; e < 256; e += blockDim.x) part[(size_t)e * gridDim.x + blockIdx.x] = tot[e];
}

template <int N>
static int zeta_blocks_impl() {
    const int lines = N * N;
    return lines < 296 ? lines : 296;
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

template <int N>
static cudaError_t zeta_impl(const float2* spec, float2* fields, const float* delta, const HarmBatch& hb,
                             const Tables& tb, double* gram_part, cudaStream_t st, const Tracer& tr) {
    using C = ZCfg<N>;
    cudaError_t e;
    if ((e = allow_smem_z(k_zeta_x<N>, C::SMEM_X)) != cudaSuccess) return e;
    if ((e = allow_smem_z(k_zeta_y<N>, C::SMEM_X)) != cudaSuccess) return e;
    if ((e = allow_smem_z(k_zeta_z_gram<N>, C::SMEM_Z)) != cudaSuccess) return e;
    dim3 g1(N / C::W, N, 1);
    tr(K_ZETA_X, 0, st);
    k_zeta_x<N><<<g1, C::TS, C::SMEM_X, st>>>(spec, fields, hb, tb);
    tr(K_ZETA_X, 1, st);
    dim3 g2(N / C::W, N, hb.S);
    tr(K_ZETA_Y, 0, st);
    k_zeta_y<N><<<g2, C::TS, C::SMEM_X, st>>>(fields, tb.tw);
    tr(K_ZETA_Y, 1, st);
    tr(K_ZETA_Z_GRAM, 0, st);
    k_zeta_z_gram<N><<<zeta_blocks_impl<N>(), C::ZT, C::SMEM_Z, st>>>(fields, hb.S, delta, tb.tw, gram_part);
    tr(K_ZETA_Z_GRAM, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_zeta_lm(int N, const float2* spec, float2* fields, const float* delta, const HarmBatch& hb,
                           const Tables& tb, double* gram_part, cudaStream_t st, const Tracer& tr) {
    if (hb.S < 1 || hb.S > 16) return cudaErrorInvalidValue;
    switch (N) {
        case 16: return zeta_impl<16>(spec, fields, delta, hb, tb, gram_part, st, tr);
        case 32: return zeta_impl<32>(spec, fields, delta, hb, tb, gram_part, st, tr);
        case 64: return zeta_impl<64>(spec, fields, delta, hb, tb, gram_part, st, tr);
        case 128: return zeta_impl<128>(spec, fields, delta, hb, tb, gram_part, st, tr);
        case 256: return zeta_impl<256>(spec, fields, delta, hb, tb, gram_part, st, tr);
        case 512: return zeta_impl<512>(spec, fields, delta, hb, tb, gram_part, st, tr);
        case 1024: return zeta_impl<1024>(spec, fields, delta, hb, tb, gram_part, st, tr);
    }
    return cudaErrorInvalidValue;
}

}  // namespace hermes
