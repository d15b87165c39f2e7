// 3-D FFT passes of the xi / xi_l path.
//
// Layouts (z fastest everywhere):
//   grid / delta : float  [N][N][N]        real field
//   spec         : float2 [N][N][N/2]      half spectrum, k_z in [0, N/2); the
//                                          Nyquist plane k_z = N/2 is not stored
//                                          because every window is zero there
//   work         : float2 [S][N][N][N/2]   filtered spectra of one window batch
//
// Forward (Sec. 2 convention, e^{-ik.x}): F1 real-to-complex along z fused with
// delta = eps / eps_bar - 1 (delta is written back in place for the final
// contraction), F2 along y, F3 along x with delta^(0) := 0.
//
// Inverse per batch of S windows (Sec. 3.5, eps_W = iFT[FT(eps) K_W]):
//   I1 along x: read delta^ once, multiply by K_s = W^_s Phi^ for every window
//      s of the batch, inverse FFT, store (the self-pair term of each window is
//      the radial contraction of the self-pair histogram, kspace.cu);
//   I2 along y (persistent blocks, next tile's loads in flight);
//   I3 complex-to-real along z fused with the cell contraction
//      sum_x delta(x) delta~_s(x) (Eq. pair-counting / Eq. 2rdEs): the filtered
//      fields never return to HBM.
#include "kernels.h"
#include "fft_core.cuh"
#include "async_copy.cuh"

#include <cuda.h>          // CUtensorMap (the encoder is reached through the runtime's driver entry point)
#include <cudaTypedefs.h>  // its function type
#include <cooperative_groups.h>
#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <initializer_list>

namespace hermes {

template <int N>
struct Cfg {
    static constexpr int H = N / 2;
    static_assert(N / 16 <= 32 || 256 / (N / 16) <= 15, "z lines of a block beyond the named barriers");
    static constexpr int W = (N >= 512) ? 8 : (N / 2 < 16 ? N / 2 : 16);  // columns per strided tile
    static constexpr int TS = (N / 8) * W;                                  // threads per strided tile
    static constexpr int MZ = N / 2;                                        // half-length z transform
    static constexpr int TZ = MZ / 8;
    static constexpr int LZ = (256 / TZ) > 0 ? (256 / TZ) : 1;              // z lines per block
    static constexpr int ZTHREADS = TZ * LZ;
    static constexpr size_t SMEM_STRIDED = (size_t)SmemStrided<W>::words(N) * sizeof(float2);
    static constexpr size_t SMEM_Z = (size_t)LZ * LinePad<MZ>::value * sizeof(float2);
    static constexpr size_t SMEM_Z3 = SMEM_Z + (size_t)2 * LZ * (N / 2) * sizeof(float2);  // + double stage
};

// Dynamic shared memory a block may use next to the kernels' static arrays.
constexpr size_t kMaxDynSmem = 220 * 1024;

// The shared-table window pass is the default; HERMES_X_GATHER=1 selects the
// per-element global gathers instead (kept for comparison).
static bool stab_x_enabled() {
    const char* env = getenv("HERMES_X_GATHER");
    return !(env && env[0] == '1');
}

// Lets `kernel` take `bytes` of dynamic shared memory.  The attribute is a property
// of the kernel shared by every host thread, so it is always set to the same value
// (kMaxDynSmem), never to the size of one launch: concurrent callers whose launches
// differ in size (the window pass stages S-dependent tables) then never undo each other.
template <class K>
static cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    if (bytes > kMaxDynSmem) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDynSmem);
}

// ---------------------------------------------------------------------------
// F1: real-to-complex along z.  A real line x_0..x_{N-1} is packed as
// z_j = x_{2j} + i x_{2j+1}, transformed with an N/2-point FFT, and split:
// X_k = E_k + e^{-2 pi i k/N} O_k, E_k = (Z_k + conj Z_{M-k})/2,
// O_k = (Z_k - conj Z_{M-k})/(2i), k = 0..N/2-1.
template <int N>
__global__ void __launch_bounds__(Cfg<N>::ZTHREADS) k_fwd_z_r2c(float* __restrict__ grid, float2* __restrict__ spec,
                                                                 const double* __restrict__ scal, int convert,
                                                                 const float2* __restrict__ tw) {
    using C = Cfg<N>;
    constexpr int M = C::MZ, T = C::TZ, LP = LinePad<M>::value;
    extern __shared__ float2 smem[];
    const int t = threadIdx.x % T, li = threadIdx.x / T;
    const size_t line = (size_t)blockIdx.x * C::LZ + li;
    const SmemZLine<M> sm{{smem + li * LP}, li};
    {  // batched launch: blockIdx.y = catalogue
        const size_t cat = blockIdx.y;
        grid += cat * N * N * N;
        spec += cat * N * N * (N / 2);
        scal += cat * SCAL_STRIDE;
    }
    float2* g = reinterpret_cast<float2*>(grid + line * N);
    const float inv_mean = convert ? (float)scal[2] : 1.0f;
    float2 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float2 e = g[t + i * T];
        if (convert) {
            e.x = fmaf(e.x, inv_mean, -1.0f);
            e.y = fmaf(e.y, inv_mean, -1.0f);
            g[t + i * T] = e;
        }
        v[i] = e;
    }
    fft_line<M, false>(v, t, tw, sm);
    sm.sync();
#pragma unroll
    for (int i = 0; i < 8; ++i) sm.st(t + i * T, v[i]);
    sm.sync();  // the partner k' = M - k lies in the same line
    float2* out = spec + line * (N / 2);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int k = t + i * T;
        const float2 zk = v[i];
        const float2 zm = cconj(sm.ld((M - k) & (M - 1)));
        const float2 e = cscale(cadd(zk, zm), 0.5f);
        const float2 d = csub(zk, zm);
        const float2 o = make_float2(0.5f * d.y, -0.5f * d.x);  // (zk - conj zm) / (2i)
        const float2 w = __ldg(tw + N + k);                       // e^{-2 pi i k / N}
        out[k] = cadd(e, cmul(w, o));
    }
}

// ---------------------------------------------------------------------------
// Strided complex FFT of length N along one axis, W adjacent columns per block.
// Element (pos, col) of block (bx, by, bz) is
//   data[bz*zstride + by*ystride + bx*W + col + pos*pos_stride].
template <int N, bool INV>
__global__ void __launch_bounds__(Cfg<N>::TS) k_strided(float2* __restrict__ data, long long pos_stride,
                                                         long long ystride, long long zstride, int zero_dc,
                                                         const float2* __restrict__ tw) {
    using C = Cfg<N>;
    constexpr int W = C::W, T = N / 8;
    extern __shared__ float2 smem[];
    const int col = threadIdx.x % W, t = threadIdx.x / W;
    float2* base = data + (size_t)blockIdx.z * zstride + (size_t)blockIdx.y * ystride + (size_t)blockIdx.x * W + col;
    float2 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = base[(size_t)(t + i * T) * pos_stride];
    fft_line<N, INV>(v, t, tw, SmemStrided<W>{smem, col});
    if (zero_dc && blockIdx.x == 0 && blockIdx.y == 0 && col == 0 && t == 0) v[0] = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 8; ++i) base[(size_t)(t + i * T) * pos_stride] = v[i];
}

// Persistent form of k_strided for long batches (the inverse y pass over S
// windows of C catalogues): each CTA walks tiles tile0, tile0 + gridDim.x, ...
// (tile = (column chunk, y, z) with the chunk fastest, as the plain grid) and
// issues the loads of its next tile before the current tile's FFT, so they are
// in flight across the shared-memory exchanges.  Tile coordinates advance by
// carries; no division in the loop.
template <int N, bool INV>
__global__ void __launch_bounds__(Cfg<N>::TS, 2) k_strided_pf(float2* __restrict__ data, int pos_stride,
                                                             int ystride, long long zstride, int nxt, int nyt,
                                                             int ntiles, const float2* __restrict__ tw) {
    constexpr int W = Cfg<N>::W, T = N / 8;
    extern __shared__ float2 smem[];
    const int col = threadIdx.x % W, t = threadIdx.x / W;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    int bx = tile % nxt, by = (tile / nxt) % nyt, bz = tile / nxt / nyt;
    const int dx = gridDim.x % nxt, dy = (gridDim.x / nxt) % nyt, dz = gridDim.x / nxt / nyt;
    auto base_of = [&](int x, int y, int z) {
        return data + (size_t)z * zstride + (size_t)y * ystride + x * W + col;
    };
    float2 v[8], vn[8];
    {
        const float2* b = base_of(bx, by, bz);
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = b[(t + i * T) * pos_stride];
    }
    for (; tile < ntiles; tile += gridDim.x) {
        int nx_ = bx + dx, ny_ = by + dy, nz_ = bz + dz;
        if (nx_ >= nxt) {
            nx_ -= nxt;
            ++ny_;
        }
        if (ny_ >= nyt) {
            ny_ -= nyt;
            ++nz_;
        }
        if (tile + (int)gridDim.x < ntiles) {
            const float2* b = base_of(nx_, ny_, nz_);
#pragma unroll
            for (int i = 0; i < 8; ++i) vn[i] = b[(t + i * T) * pos_stride];
        }
        fft_line<N, INV, true>(v, t, tw, SmemStrided<W>{smem, col});
        float2* b = base_of(bx, by, bz);
#pragma unroll
        for (int i = 0; i < 8; ++i) b[(t + i * T) * pos_stride] = v[i];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = vn[i];
        bx = nx_;
        by = ny_;
        bz = nz_;
    }
}

// ---------------------------------------------------------------------------
// The inverse y pass at 16 or 32 values per thread: a 256-point line needs one
// shared-memory exchange instead of two, a 1024-point line two instead of three,
// for more registers per thread.  Two forms over the tiles of k_strided_pf:
//   k_strided_e   : one tile per block, stage twiddles read from the table;
//   k_strided_pf_e: persistent blocks, the next tile's loads in flight during the
//                   transform, the thread's stage twiddles held in registers.
// The tile layout skews P slots after every 2^SH rows (chosen per shape for the
// fewest shared-memory wavefronts).
template <int N, int E, int W, int SH, int P>
__global__ void __launch_bounds__((N / E) * W) k_strided_e(float2* __restrict__ data, int pos_stride, int ystride,
                                                           long long zstride, const float2* __restrict__ tw) {
    constexpr int T = N / E;
    extern __shared__ float2 smem[];
    const int col = threadIdx.x % W, t = threadIdx.x / W;
    float2* b = data + (size_t)blockIdx.z * zstride + (size_t)blockIdx.y * ystride + blockIdx.x * W + col;
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = b[(t + i * T) * pos_stride];
    fft_line_e<N, E, true>(v, t, tw, SmemStridedSk<W, SH, P>{smem, col});
#pragma unroll
    for (int i = 0; i < E; ++i) b[(t + i * T) * pos_stride] = v[i];
}

// The inverse y pass of fields [f][x][y][z] with Z values along z (the window work
// buffer: Z = N/2; the zeta_l harmonic fields: Z = N) as k_strided_e with the strides
// fixed at compile time: the E element offsets of a thread are immediates of one base
// address instead of E computed addresses, which leaves the registers for the
// transform (MINB blocks per SM).  Grid (Z / W, N, fields).
// PAIRED: the input is in the paired order the mirror-line window passes write (16-column
// groups; in group g, line 2p + h holds columns 16g + 8h .. 16g + 8h + 7 of rows p and
// N - p interleaved, (row p, row N - p) per column, and line h of pair 0 rows 0 and N/2),
// so that those passes store whole 128-byte lines; the tile of a block covers the same
// addresses in both orders, so it is read in the paired order and written in the plain one
// in place.  Rows t + iT with iT < N/2 sit in the first slot of pair t + iT, the others in
// the second slot of pair N - t - iT (pair 0 for the row N/2).
template <int N, int Z, int E, int W, int SH, int P, int MINB, bool PAIRED = false>
__global__ void __launch_bounds__((N / E) * W, MINB) k_inv_y_e(float2* __restrict__ data,
                                                               const float2* __restrict__ tw) {
    constexpr int T = N / E;
    static_assert(!PAIRED || W == 16, "the paired order is laid out in 16-column groups");
    extern __shared__ float2 smem[];
    const int col = threadIdx.x % W, t = threadIdx.x / W;
    float2* b = data + (size_t)blockIdx.z * N * N * Z + (size_t)blockIdx.y * N * Z + blockIdx.x * W + col + t * Z;
    float2 v[E];
    if constexpr (PAIRED) {
        const float2* plane = data + (size_t)blockIdx.z * N * N * Z + (size_t)blockIdx.y * N * Z + blockIdx.x * W;
        const int h = col >> 3, c2 = 2 * (col & 7);
        const float2* pa = plane + (size_t)(2 * t + h) * Z + c2;              // row t + iT: line 2(t + iT) + h
        const float2* pb = plane + (size_t)(2 * N - 2 * t + h) * Z + c2 + 1;  // line 2(N - t - iT) + h
        const size_t nyq = t == 0 ? (size_t)N * Z : 0;                        // row N/2: line h of pair 0
#pragma unroll
        for (int i = 0; i < E / 2; ++i) v[i] = pa[(size_t)i * 2 * T * Z];
#pragma unroll
        for (int i = E / 2; i < E; ++i) v[i] = *(pb - (size_t)i * 2 * T * Z - (i == E / 2 ? nyq : 0));
    } else {
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = b[i * T * Z];
    }
    fft_line_e<N, E, true>(v, t, tw, SmemStridedSk<W, SH, P>{smem, col});
#pragma unroll
    for (int i = 0; i < E; ++i) b[i * T * Z] = v[i];
}

template <int N, int E, int W, int SH, int P, int MINB>
__global__ void __launch_bounds__((N / E) * W, MINB) k_strided_pf_e(float2* __restrict__ data, int pos_stride,
                                                                    int ystride, long long zstride, int nxt, int nyt,
                                                                    int ntiles, const float2* __restrict__ tw) {
    constexpr int T = N / E;
    extern __shared__ float2 smem[];
    const int col = threadIdx.x % W, t = threadIdx.x / W;
    int tile = blockIdx.x;
    if (tile >= ntiles) return;
    float2 wc[stage_twiddle_count<N, E>() + 1];
    load_stage_twiddles_e<N, E, true>(t, tw, wc);
    int bx = tile % nxt, by = (tile / nxt) % nyt, bz = tile / nxt / nyt;
    const int dx = gridDim.x % nxt, dy = (gridDim.x / nxt) % nyt, dz = gridDim.x / nxt / nyt;
    auto base_of = [&](int x, int y, int z) {
        return data + (size_t)z * zstride + (size_t)y * ystride + x * W + col;
    };
    float2 v[E], vn[E];
    {
        const float2* b = base_of(bx, by, bz);
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = b[(t + i * T) * pos_stride];
    }
    for (; tile < ntiles; tile += gridDim.x) {
        int nx_ = bx + dx, ny_ = by + dy, nz_ = bz + dz;
        if (nx_ >= nxt) {
            nx_ -= nxt;
            ++ny_;
        }
        if (ny_ >= nyt) {
            ny_ -= nyt;
            ++nz_;
        }
        if (tile + (int)gridDim.x < ntiles) {
            const float2* b = base_of(nx_, ny_, nz_);
#pragma unroll
            for (int i = 0; i < E; ++i) vn[i] = b[(t + i * T) * pos_stride];
        }
        fft_line_e_wc<N, E, true>(v, t, tw, SmemStridedSk<W, SH, P>{smem, col}, wc);
        float2* b = base_of(bx, by, bz);
#pragma unroll
        for (int i = 0; i < E; ++i) b[(t + i * T) * pos_stride] = v[i];
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = vn[i];
        bx = nx_;
        by = ny_;
        bz = nz_;
    }
}

// Legendre polynomial L_l(mu) by the three-term recurrence.
__device__ __forceinline__ float legendre(int ell, float mu) {
    if (ell == 0) return 1.0f;
    float p0 = 1.0f, p1 = mu;
    for (int n = 1; n < ell; ++n) {
        const float p2 = ((float)(2 * n + 1) * mu * p1 - (float)n * p0) / (float)(n + 1);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// cos(2 pi j / N) from the twiddle table.
template <int N>
__device__ __forceinline__ float cos_tab(const float2* __restrict__ tw, int j) {
    return __ldg(tw + N + (j & (N - 1))).x;
}

// ---------------------------------------------------------------------------
// I1: first inverse pass (along x) with the window multiply of a batch of S
// windows fused in: K_s(n) = scale * T_s(|n|^2) * Phi^(n) * L_l(k_z/k), all
// windows of the batch sharing the order l (Phi^, L_l and scale are applied to
// the input once); for axisymmetric windows K_s(n) = T_perp_s(n_x^2 + n_y^2) *
// T_par_j(|n_z|) * Phi^(n), the batch sharing the line-of-sight bin j.  The
// self-pair term of each window is not summed here: it is the radial
// contraction of the self-pair histogram (kspace.cu).
//
// STAB: the block first copies the radial factors it needs into shared memory
// (its columns see |n|^2 = a^2 + n_y^2 + n_z^2 for a = |n_x| only, so H rows per
// column cover every element, the +-n_x pair included), with asynchronous
// 16-byte copies issued before the spectrum is read; otherwise every element
// gathers them from the global table (16-byte loads of 4 bins).

// Row stride (floats) of the shared radial table: S rounded up to 4, plus 4
// when that is a multiple of 8, so the 16-byte reads of a warp (32 rows at
// consecutive (|n_x|, column)) spread over all banks.
__host__ __device__ constexpr int stab_row_stride(int S) {
    return ((S + 3) & ~3) + ((((S + 3) >> 2) & 1) ? 0 : 4);
}

template <int N, bool STAB>
__global__ void __launch_bounds__(Cfg<N>::TS, 1) k_inv_x_window(const float2* __restrict__ spec,
                                                              float2* __restrict__ work, const WinBatch wb,
                                                              const Tables tb) {
    using C = Cfg<N>;
    constexpr int W = C::W, T = N / 8, H = N / 2;
    extern __shared__ __align__(16) float2 smem[];
    float* ttab = reinterpret_cast<float*>(smem + SmemStrided<W>::words(N));  // [a][col][RS] (STAB)
    const int RS = stab_row_stride(wb.S);
    const int col = threadIdx.x % W, t = threadIdx.x / W;
    const int ky = blockIdx.y, kz = blockIdx.x * W + col;
    const size_t xstride = (size_t)N * H;
    {  // batched launch: blockIdx.z = catalogue
        const size_t cat = blockIdx.z;
        spec += cat * N * N * H;
        work += cat * wb.S * N * N * H;
    }
    const int ny = signed_freq(ky, N), nz = kz;
    const bool nyq_y = (ky == H);
    if constexpr (STAB) {
        // rows of S4 16-byte pieces per (a, column); consecutive threads copy one row's pieces
        const int S4 = (wb.S + 3) >> 2;
        const int total = H * W * S4;
        const int ny2 = nyq_y ? 0 : ny * ny;
        for (int e = threadIdx.x; e < total; e += C::TS) {
            const int s4 = e % S4, c = (e / S4) % W, a = e / (S4 * W);
            const int nzc = blockIdx.x * W + c;
            const int qq = nyq_y ? 0 : a * a + ny2 + (wb.cyl ? 0 : nzc * nzc);
            ac::cp_async16(ttab + (a * W + c) * RS + 4 * s4,
                           reinterpret_cast<const float4*>(wb.tab + (size_t)qq * wb.nbp) + s4);
        }
        ac::cp_async_commit();
    }
    const float2* src = spec + (size_t)ky * H + kz;
    float2 v0[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v0[i] = src[(size_t)(t + i * T) * xstride];
    // Phi^, the Nyquist mask, scale and L_l(k_z/k) are folded into the input once,
    // so per window v = v0 * T_s(|n|^2)
    const float phyz = __ldg(tb.phi + ky) * __ldg(tb.phi + kz);
    int q[8];  // |n|^2 (gather form only)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int kx = t + i * T;
        const int nx = signed_freq(kx, N);
        const bool nyq = nyq_y || (kx == H);
        const int qi = nyq ? 0 : nx * nx + ny * ny + nz * nz;  // table index stays in range on Nyquist lanes
        const float ph = nyq ? 0.0f : __ldg(tb.phi + kx) * phyz;
        // the window's factor that does not depend on the bin: scale * L_l(k_z/k), or T_par_j(|n_z|)
        // (ring windows apply their own line-of-sight factor per window below)
        const float a = wb.cyl ? (wb.par_stride ? 1.0f : __ldg(wb.par + nz))
                               : wb.scale * legendre(wb.ell, qi > 0 ? (float)nz * rsqrtf((float)qi) : 0.0f);
        v0[i] = cscale(v0[i], ph * a);
        q[i] = (wb.cyl && !nyq) ? nx * nx + ny * ny : qi;
    }
    // Under STAB the row of element i is |n_x| = t + iT (i < 4) or N - t - iT (i >= 4; the
    // Nyquist element t = 0, i = 4 reads row 0): two per-thread bases and constant steps,
    // so the offsets need no registers of their own.
    const int qlo = (t * W + col) * RS, qhi = ((N - t) * W + col) * RS;
    auto trow = [&](int i) {
        return i < 4 ? qlo + i * (T * W) * RS : ((t == 0 && i == 4) ? col * RS : qhi - i * (T * W) * RS);
    };
    if constexpr (STAB) {
        ac::cp_async_wait_all();
        __syncthreads();
    }
    float2 wc[3 * twiddled_stages<N>()];  // the thread's stage twiddles, the same for every window
    load_stage_twiddles<N, true>(t, tb.tw, wc);
    const int nbp = wb.nbp;
    for (int g = 0; g < wb.S; g += 4) {
        // radial factors of windows g..g+3 at every element: one 16-byte load each
        float4 tv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            tv[i] = STAB ? *reinterpret_cast<const float4*>(ttab + trow(i) + g)
                         : __ldg(reinterpret_cast<const float4*>(wb.tab + (size_t)q[i] * nbp + g));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int s = g + j;
            if (s >= wb.S) break;  // uniform across the block
            // ring windows: this window's line-of-sight factor at the thread's |n_z|
            const float pz = wb.par_stride ? __ldg(wb.par + (size_t)s * wb.par_stride + nz) : 1.0f;
            float2 v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                v[i] = cscale(v0[i], pz * (j == 0 ? tv[i].x : (j == 1 ? tv[i].y : (j == 2 ? tv[i].z : tv[i].w))));
            fft_line_wc<N, true>(v, t, tb.tw, SmemStrided<W>{smem, col}, wc);
            float2* dst = work + (size_t)s * N * N * H + (size_t)ky * H + kz;
#pragma unroll
            for (int i = 0; i < 8; ++i) dst[(size_t)(t + i * T) * xstride] = v[i];
        }
    }
}

// The window pass with two windows in flight per thread: windows s and s + 1 are
// scaled, transformed and stored together, their transforms exchanging through two
// tile buffers behind the same barriers (half the barriers per window and twice the
// independent instructions between them).  The radial table is staged as in
// k_inv_x_window but with rows of RS = 4, 8 or 16 floats and no padding: the
// 16-byte chunk j of row r sits at chunk j ^ ((r >> rsh) & (RS / 4 - 1)), so the
// 16-byte reads of a quarter warp (8 consecutive rows) meet 8 distinct bank groups.
// Used when the table of the batch (S <= 16) and two tiles fit in shared memory.
__host__ __device__ constexpr int pair_row_floats(int S) { return S <= 4 ? 4 : (S <= 8 ? 8 : 16); }

template <int N>
__global__ void __launch_bounds__(Cfg<N>::TS, 1) k_inv_x_window_pair(const float2* __restrict__ spec,
                                                                   float2* __restrict__ work, const WinBatch wb,
                                                                   const Tables tb) {
    using C = Cfg<N>;
    constexpr int W = C::W, T = N / 8, H = N / 2;
    constexpr int TILE = SmemStrided<W>::words(N);
    extern __shared__ __align__(16) float2 smem[];
    float* ttab = reinterpret_cast<float*>(smem + 2 * TILE);  // [a][col][RS], chunks swizzled
    const int RS = pair_row_floats(wb.S);
    const int rsh = RS == 16 ? 1 : 2, cmask = RS / 4 - 1;
    const int col = threadIdx.x % W, t = threadIdx.x / W;
    const int ky = blockIdx.y, kz = blockIdx.x * W + col;
    const size_t xstride = (size_t)N * H;
    {  // batched launch: blockIdx.z = catalogue
        const size_t cat = blockIdx.z;
        spec += cat * N * N * H;
        work += cat * wb.S * N * N * H;
    }
    const int ny = signed_freq(ky, N), nz = kz;
    const bool nyq_y = (ky == H);
    {
        const int S4 = (wb.S + 3) >> 2;
        const int total = H * W * S4;
        const int ny2 = nyq_y ? 0 : ny * ny;
        for (int e = threadIdx.x; e < total; e += C::TS) {
            const int s4 = e % S4, c = (e / S4) % W, a = e / (S4 * W);
            const int nzc = blockIdx.x * W + c;
            const int qq = nyq_y ? 0 : a * a + ny2 + (wb.cyl ? 0 : nzc * nzc);
            const int row = a * W + c;
            ac::cp_async16(ttab + row * RS + 4 * (s4 ^ ((row >> rsh) & cmask)),
                           reinterpret_cast<const float4*>(wb.tab + (size_t)qq * wb.nbp) + s4);
        }
        ac::cp_async_commit();
    }
    const float2* src = spec + (size_t)ky * H + kz;
    float2 v0[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v0[i] = src[(size_t)(t + i * T) * xstride];
    const float phyz = __ldg(tb.phi + ky) * __ldg(tb.phi + kz);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int kx = t + i * T;
        const int nx = signed_freq(kx, N);
        const bool nyq = nyq_y || (kx == H);
        const int qi = nyq ? 0 : nx * nx + ny * ny + nz * nz;
        const float ph = nyq ? 0.0f : __ldg(tb.phi + kx) * phyz;
        const float a = wb.cyl ? (wb.par_stride ? 1.0f : __ldg(wb.par + nz))
                               : wb.scale * legendre(wb.ell, qi > 0 ? (float)nz * rsqrtf((float)qi) : 0.0f);
        v0[i] = cscale(v0[i], ph * a);
    }
    // table row of element i: |n_x| = t + iT (i < 4) or N - t - iT (i >= 4; the Nyquist
    // element t = 0, i = 4 is zero and reads row 0)
    auto trow = [&](int i) {
        const int ax = i < 4 ? t + i * T : ((t == 0 && i == 4) ? 0 : N - t - i * T);
        return ax * W + col;
    };
    ac::cp_async_wait_all();
    __syncthreads();
    float2 wc[3 * twiddled_stages<N>()];
    load_stage_twiddles<N, true>(t, tb.tw, wc);
    const SmemStrided<W> sms[2] = {{smem, col}, {smem + TILE, col}};
    for (int g = 0; g < wb.S; g += 4) {
        float4 tv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = trow(i);
            tv[i] = *reinterpret_cast<const float4*>(ttab + r * RS + 4 * ((g >> 2) ^ ((r >> rsh) & cmask)));
        }
#pragma unroll
        for (int jp = 0; jp < 4; jp += 2) {
            const int s = g + jp;
            if (s >= wb.S) break;  // uniform across the block
            const bool two = s + 1 < wb.S;
            const float pz0 = wb.par_stride ? __ldg(wb.par + (size_t)s * wb.par_stride + nz) : 1.0f;
            const float pz1 = (wb.par_stride && two) ? __ldg(wb.par + (size_t)(s + 1) * wb.par_stride + nz) : 1.0f;
            float2 v[2][8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float f0 = jp == 0 ? tv[i].x : tv[i].z, f1 = jp == 0 ? tv[i].y : tv[i].w;
                v[0][i] = cscale(v0[i], pz0 * f0);
                v[1][i] = cscale(v0[i], pz1 * f1);
            }
            fft_lines_wc<N, true, 2>(v, t, sms, wc);
            float2* dst = work + (size_t)s * N * N * H + (size_t)ky * H + kz;
#pragma unroll
            for (int i = 0; i < 8; ++i) dst[(size_t)(t + i * T) * xstride] = v[0][i];
            if (two) {
                dst += (size_t)N * N * H;
#pragma unroll
                for (int i = 0; i < 8; ++i) dst[(size_t)(t + i * T) * xstride] = v[1][i];
            }
        }
    }
}

// The window pass on mirror lines: the x lines at k_y and N - k_y (same n_y^2, same
// Phi^(k_y)) see the same radial factor at every element, so a block transforms both for
// its W columns, their FFTs exchanging through two tiles behind the same barriers, and one
// table read serves the two lines (the table as in k_inv_x_window_pair).  Blocks at
// k_y = 0 and N/2 (their own mirrors) transform one line set.
// ONE: each window's factors are read from the table when that window is scaled (8 scalar
// loads, 4-way bank conflicts) instead of four windows' factors held in 32 registers; at 128
// registers a thread that frees them stops spilling, and the spill reloads were a large part
// of the pass's long-scoreboard stalls.
// PAIRED (8-column tiles): the two lines' values of a column are stored side by side, one
// 16-byte store per element, in the paired order that k_inv_y_e<..., PAIRED> reads, so
// that every store instruction writes whole 128-byte lines (8-column tiles of the plain
// order write half lines); grid (N / 2 / W, N / 2): the block at k_y = 0 also writes the
// k_y = N/2 line, which is zero.
// TMA (paired order only): each window's tile goes out as two tiled bulk stores through the
// tensor map tmap (a 3-D view of the work buffer: float32 along k_z, the N lines of an x
// plane, x planes of every window), staged densely ([x][8 columns][two lines]) over the
// FFT's two exchange tiles once the last exchange has been read; the next window's first
// exchange waits until the stores have read the stage.  The threads' stores become shared
// stores; the DRAM writes leave the SM as 32 KB boxes.
template <int N, bool ONE = false, bool PAIRED = false, bool TMA = false>
__global__ void __launch_bounds__(Cfg<N>::TS, 1) k_inv_x_window_mirror(const float2* __restrict__ spec,
                                                                     float2* __restrict__ work, const WinBatch wb,
                                                                     const Tables tb,
                                                                     const __grid_constant__ CUtensorMap tmap) {
    using C = Cfg<N>;
    constexpr int W = C::W, T = N / 8, H = N / 2;
    static_assert(!PAIRED || W == 8, "the paired order pairs two 8-column tiles in a 16-column group");
    static_assert(!TMA || (PAIRED && N == 512), "tiled bulk stores of the paired order at 512^3");
    static_assert(!TMA || 2 * SmemStrided<W>::words(N) >= N * 2 * W, "the stage fits in the two exchange tiles");
    constexpr int TILE = SmemStrided<W>::words(N);
    extern __shared__ __align__(16) float2 smem[];
    float* ttab = reinterpret_cast<float*>(smem + 2 * TILE);  // [a][col][RS], chunks swizzled
    const int RS = pair_row_floats(wb.S);
    const int rsh = RS == 16 ? 1 : 2, cmask = RS / 4 - 1;
    const int col = threadIdx.x % W, t = threadIdx.x / W;
    const int ky = blockIdx.y, kyb = (N - ky) & (N - 1), kz = blockIdx.x * W + col;  // blockIdx.y in [0, H]
    const bool two = (ky != 0 && ky != H);
    const size_t xstride = (size_t)N * H;
    {  // batched launch: blockIdx.z = catalogue
        const size_t cat = blockIdx.z;
        spec += cat * N * N * H;
        work += cat * wb.S * N * N * H;
    }
    const int ny = signed_freq(ky, N), nz = kz;
    const bool nyq_y = (ky == H);
    {
        const int S4 = (wb.S + 3) >> 2;
        const int total = H * W * S4;
        const int ny2 = nyq_y ? 0 : ny * ny;
        for (int e = threadIdx.x; e < total; e += C::TS) {
            const int s4 = e % S4, c = (e / S4) % W, a = e / (S4 * W);
            const int nzc = blockIdx.x * W + c;
            const int qq = nyq_y ? 0 : a * a + ny2 + (wb.cyl ? 0 : nzc * nzc);
            const int row = a * W + c;
            ac::cp_async16(ttab + row * RS + 4 * (s4 ^ ((row >> rsh) & cmask)),
                           reinterpret_cast<const float4*>(wb.tab + (size_t)qq * wb.nbp) + s4);
        }
        ac::cp_async_commit();
    }
    const float2* srca = spec + (size_t)ky * H + kz;
    const float2* srcb = spec + (size_t)kyb * H + kz;
    float2 va0[8], vb0[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        va0[i] = srca[(size_t)(t + i * T) * xstride];
        vb0[i] = two ? srcb[(size_t)(t + i * T) * xstride] : make_float2(0.f, 0.f);
    }
    const float phyz = __ldg(tb.phi + ky) * __ldg(tb.phi + kz);  // Phi^(N - k_y) = Phi^(k_y)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int kx = t + i * T;
        const int nx = signed_freq(kx, N);
        const bool nyq = nyq_y || (kx == H);
        const int qi = nyq ? 0 : nx * nx + ny * ny + nz * nz;
        const float ph = nyq ? 0.0f : __ldg(tb.phi + kx) * phyz;
        const float a = wb.cyl ? (wb.par_stride ? 1.0f : __ldg(wb.par + nz))
                               : wb.scale * legendre(wb.ell, qi > 0 ? (float)nz * rsqrtf((float)qi) : 0.0f);
        va0[i] = cscale(va0[i], ph * a);
        vb0[i] = cscale(vb0[i], ph * a);
    }
    auto trow = [&](int i) {
        const int ax = i < 4 ? t + i * T : ((t == 0 && i == 4) ? 0 : N - t - i * T);
        return ax * W + col;
    };
    ac::cp_async_wait_all();
    __syncthreads();
    float2 wc[3 * twiddled_stages<N>()];
    load_stage_twiddles<N, true>(t, tb.tw, wc);
    const SmemStrided<W> sms[2] = {{smem, col}, {smem + TILE, col}};
    const int cat = blockIdx.z;
    for (int g = 0; g < wb.S; g += 4) {
        float4 tv[ONE ? 1 : 8];
        if constexpr (!ONE) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = trow(i);
                tv[i] = *reinterpret_cast<const float4*>(ttab + r * RS + 4 * ((g >> 2) ^ ((r >> rsh) & cmask)));
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int s = g + j;
            if (s >= wb.S) break;  // uniform across the block
            const float pz = wb.par_stride ? __ldg(wb.par + (size_t)s * wb.par_stride + nz) : 1.0f;
            float2 v[2][8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                float f;
                if constexpr (ONE) {
                    const int r = trow(i);
                    f = pz * ttab[r * RS + 4 * ((g >> 2) ^ ((r >> rsh) & cmask)) + j];
                } else {
                    f = pz * (j == 0 ? tv[i].x : (j == 1 ? tv[i].y : (j == 2 ? tv[i].z : tv[i].w)));
                }
                v[0][i] = cscale(va0[i], f);
                v[1][i] = cscale(vb0[i], f);
            }
            if constexpr (TMA) {  // the previous window's stores have read the stage before its first exchange
                if (threadIdx.x == 0) ac::bulk_wait_read_all();
            }
            fft_lines_wc<N, true, 2>(v, t, sms, wc);
            if constexpr (TMA) {
                __syncthreads();  // every thread has read the last exchange
                float4* stg = reinterpret_cast<float4*>(smem);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    stg[(t + i * T) * W + col] = make_float4(v[0][i].x, v[0][i].y, v[1][i].x, v[1][i].y);
                ac::fence_proxy_async();
                __syncthreads();
                if (threadIdx.x == 0) {
                    const int c0 = 32 * (int)(blockIdx.x >> 1), c1 = 2 * ky + (int)(blockIdx.x & 1);
                    const int c2 = (cat * wb.S + s) * N;
                    ac::tma_store_3d(&tmap, smem, c0, c1, c2);
                    ac::tma_store_3d(&tmap, smem + (N / 2) * 2 * W, c0, c1, c2 + N / 2);
                    ac::bulk_commit();
                }
            } else if constexpr (PAIRED) {
                // line 2 k_y + (tile & 1) of 16-column group tile / 2, slots (k_y, N - k_y) of column col
                const int off = t * (N * H) + (2 * ky + (int)(blockIdx.x & 1)) * H + (int)(blockIdx.x >> 1) * 16 + 2 * col;
                float2* dst = work + (size_t)s * N * N * H + off;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    *reinterpret_cast<float4*>(dst + (size_t)i * T * N * H) =
                        make_float4(v[0][i].x, v[0][i].y, v[1][i].x, v[1][i].y);
            } else {
                float2* dst = work + (size_t)s * N * N * H + (size_t)kz;
#pragma unroll
                for (int i = 0; i < 8; ++i) dst[(size_t)(t + i * T) * xstride + (size_t)ky * H] = v[0][i];
                if (two) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) dst[(size_t)(t + i * T) * xstride + (size_t)kyb * H] = v[1][i];
                }
            }
        }
    }
    if constexpr (TMA) {  // the stage stays valid until the last stores have completed
        if (threadIdx.x == 0) ac::bulk_wait_all();
    }
}

// ---------------------------------------------------------------------------
// I3: complex-to-real along z fused with the cell contraction.
// Z'_k = (X_k + conj X_{M-k}) + i e^{+2 pi i k/N} (X_k - conj X_{M-k}), X_M = 0;
// z = IFFT_M(Z') gives x_{2j} = Re z_j, x_{2j+1} = Im z_j (unnormalised).
template <int N>
__global__ void __launch_bounds__(Cfg<N>::ZTHREADS, 3) k_inv_z_c2r_contract(const float2* __restrict__ work, int S,
                                                                             const float* __restrict__ delta,
                                                                             const float2* __restrict__ tw,
                                                                             double* __restrict__ dd_part,
                                                                             unsigned* __restrict__ err) {
    using C = Cfg<N>;
    constexpr int M = C::MZ, T = C::TZ, LP = LinePad<M>::value, H = N / 2, LZ = C::LZ;
    constexpr int NW = C::ZTHREADS / 32;
    constexpr uint32_t STAGE = (uint32_t)(LZ * H * sizeof(float2));  // the block's LZ lines of one window
    // Window s+1 is fetched by one bulk copy (the LZ lines are contiguous) into
    // the other half of a double buffer while window s is transformed.
    extern __shared__ __align__(16) float2 smem[];
    float2* stage = smem;                  // [2][LZ * H], dense
    float2* lines = smem + 2 * LZ * H;     // LZ padded lines for the FFT exchanges
    __shared__ __align__(8) uint64_t full[2];
    __shared__ float wdd[NW][MAX_BATCH];
    const int t = threadIdx.x % T, li = threadIdx.x / T;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t line0 = (size_t)blockIdx.x * LZ;
    const size_t line = line0 + li;
    const SmemZLine<M> sm{{lines + li * LP}, li};
    {  // batched launch: blockIdx.y = catalogue
        const size_t cat = blockIdx.y;
        work += cat * S * N * N * H;
        delta += cat * N * N * N;
        dd_part += cat * S * gridDim.x;
    }
    if (threadIdx.x == 0) {
        ac::mbar_init(&full[0], 1);
        ac::mbar_init(&full[1], 1);
        ac::mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && S > 0) {
        ac::mbar_expect_tx(&full[0], STAGE);
        ac::bulk_g2s(stage, work + line0 * H, STAGE, &full[0]);
    }
    const float2* dl = reinterpret_cast<const float2*>(delta + line * N);
    float2 wc[3 * twiddled_stages<M>() + 1];  // the thread's stage twiddles (+1: M = 8 has none)
    load_stage_twiddles<M, true>(t, tw, wc);
    float2 d2[8], wk[8];  // the thread's delta pairs and split twiddles e^{+2 pi i k / N}, k = t + iT
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        d2[i] = dl[t + i * T];
        wk[i] = cconj(__ldg(tw + N + t + i * T));
    }
    bool late = false;
    for (int s = 0; s < S; ++s) {
        __syncthreads();  // every thread is done with the buffer that the next copy overwrites
        if (threadIdx.x == 0 && s + 1 < S) {
            ac::fence_proxy_async();
            ac::mbar_expect_tx(&full[(s + 1) & 1], STAGE);
            ac::bulk_g2s(stage + ((s + 1) & 1) * LZ * H, work + (size_t)(s + 1) * N * N * H + line0 * H, STAGE,
                         &full[(s + 1) & 1]);
        }
        if (!ac::mbar_wait(&full[s & 1], (s >> 1) & 1)) late = true;
        const float2* X = stage + (s & 1) * LZ * H + li * H;
        float2 v[8], xm[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = X[t + i * T];
        // the partner X_{M-k} of element k = t + iT comes from the stage too (a warp's reads are
        // one contiguous descending run; X_M = 0); this beats 16 warp shuffles
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = t + i * T;
            xm[i] = (k == 0) ? make_float2(0.f, 0.f) : X[M - k];
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float2 xk = v[i];
            const float2 xc = cconj(xm[i]);
            const float2 a = cadd(xk, xc);
            const float2 c = cmul(wk[i], csub(xk, xc));
            v[i] = make_float2(a.x - c.y, a.y + c.x);
        }
        fft_line_wc<M, true>(v, t, tw, sm, wc);
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) acc = fmaf(d2[i].x, v[i].x, fmaf(d2[i].y, v[i].y, acc));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) wdd[wid][s] = acc;
    }
    if (late) atomicOr(err, 4u);
    __syncthreads();
    if (threadIdx.x < S) {
        double tot = 0.0;
        for (int w = 0; w < NW; ++w) tot += (double)wdd[w][threadIdx.x];
        dd_part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = tot;
    }
}

// I3 at 16 values per thread: a half-length line (N/2 points) is held by N/32
// threads, so one shared-memory exchange replaces two at N = 512 (256 = 16 x 16);
// two lines share a warp.  LZ = THREADS / (N/32) lines per block, their windows
// staged by bulk copies as in k_inv_z_c2r_contract; a block covering SLOTS blocks
// of that kernel writes its sum into the first of their partial slots and 0 into
// the others, so the partials keep the layout of the radix-8 form.  The stage
// twiddles and the c2r split twiddles are held in registers.
// Shared-memory pitches of the 16-value contraction pass: SP float2 per staged line (N/2:
// dense, one bulk copy per window; more: one copy per line) and the exchange lines (one pad
// slot every 2^SH elements, LP float2 per line).  At 256^3 four 128-point lines share a warp:
// the dense stage and one pad per 16 put the two lines of a half warp on the same banks,
// and these pitches reach the minimum wavefronts (bank simulation of every access).
template <int N>
struct Z16Pitch {
    static constexpr int SP = N / 2, SH = line_shift(N / 2), LP = LinePad<N / 2>::value;
};
template <>
struct Z16Pitch<256> {
    static constexpr int SP = 136, SH = 3, LP = 152;
};
template <int SH>
struct SmemWarpLineSh {  // a padded line whose threads all belong to one warp
    float2* p;
    __device__ __forceinline__ static int at(int pos) { return pos + (pos >> SH); }
    __device__ __forceinline__ float2 ld(int pos) const { return p[at(pos)]; }
    __device__ __forceinline__ void st(int pos, float2 v) const { p[at(pos)] = v; }
    __device__ __forceinline__ static void sync() { __syncwarp(); }
};

template <int N, int THREADS>
struct Z16Cfg {
    static constexpr int M = N / 2, E = 16, T = M / E, LZ = THREADS / T;
    static constexpr int SP = Z16Pitch<N>::SP, SH = Z16Pitch<N>::SH, LP = Z16Pitch<N>::LP;
    static_assert(((M - 1) + ((M - 1) >> SH)) < LP && SP >= M && (SP * 8) % 16 == 0, "line pitches");
    static constexpr int SLOTS = LZ / Cfg<N>::LZ;  // partial slots of the radix-8 layout per block
    static_assert(SLOTS >= 1 && SLOTS * Cfg<N>::LZ == LZ, "blocks cover whole radix-8 blocks");
    static constexpr size_t SMEM = (size_t)2 * LZ * SP * sizeof(float2) + (size_t)LZ * LP * sizeof(float2);
};

template <int N, int THREADS, int MINB, bool WKS = false>
__global__ void __launch_bounds__(THREADS, MINB) k_inv_z_c2r_contract_e16(const float2* __restrict__ work, int S,
                                                                       const float* __restrict__ delta,
                                                                       const float2* __restrict__ tw,
                                                                       double* __restrict__ dd_part,
                                                                       unsigned* __restrict__ err) {
    using C = Z16Cfg<N, THREADS>;
    constexpr int M = C::M, E = C::E, T = C::T, LZ = C::LZ, LP = C::LP, SP = C::SP, H = N / 2;
    constexpr int SLOTS = C::SLOTS;
    static_assert(T <= 32 && 32 % T == 0, "lines within a warp");
    constexpr int NW = THREADS / 32;
    constexpr uint32_t STAGE = (uint32_t)(LZ * H * sizeof(float2));  // bytes per window
    extern __shared__ __align__(16) float2 smem[];
    float2* stage = smem;
    float2* lines = smem + 2 * LZ * SP;
    __shared__ __align__(8) uint64_t full[2];
    __shared__ float wdd[NW][MAX_BATCH];
    const int t = threadIdx.x % T, li = threadIdx.x / T;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t line0 = (size_t)blockIdx.x * LZ;
    const size_t line = line0 + li;
    const SmemWarpLineSh<C::SH> sm{lines + li * LP};  // the T <= 32 threads of a line share a warp
    // window w's LZ lines into stage buffer b: one bulk copy (dense) or one per line (pitch SP)
    auto fetch = [&](int w, int b) {
        const float2* src = work + (size_t)w * N * N * H + line0 * H;
        float2* dst = stage + b * LZ * SP;
        ac::mbar_expect_tx(&full[b], STAGE);
        if constexpr (SP == H) {
            ac::bulk_g2s(dst, src, STAGE, &full[b]);
        } else {
#pragma unroll 1
            for (int l = 0; l < LZ; ++l)
                ac::bulk_g2s(dst + l * SP, src + (size_t)l * H, (uint32_t)(H * sizeof(float2)), &full[b]);
        }
    };
    {  // batched launch: blockIdx.y = catalogue
        const size_t cat = blockIdx.y;
        work += cat * S * N * N * H;
        delta += cat * N * N * N;
        dd_part += cat * S * (SLOTS * gridDim.x);  // partial layout of the radix-8 form
    }
    if (threadIdx.x == 0) {
        ac::mbar_init(&full[0], 1);
        ac::mbar_init(&full[1], 1);
        ac::mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0 && S > 0) fetch(0, 0);
    const float2* dl = reinterpret_cast<const float2*>(delta + line * N);
    float2 d2[E];
#pragma unroll
    for (int i = 0; i < E; ++i) d2[i] = dl[t + i * T];
    // the c2r split twiddles e^{+2 pi i k / N}, k = t + iT: in registers, or (WKS) in a table
    // shared by the block and read per window (32 registers fewer)
    __shared__ float2 swk[WKS ? M : 1];
    float2 wk[WKS ? 1 : E];
    if constexpr (WKS) {
        for (int k = threadIdx.x; k < M; k += THREADS) swk[k] = cconj(__ldg(tw + N + k));
    } else {
#pragma unroll
        for (int i = 0; i < E; ++i) wk[i] = cconj(__ldg(tw + N + t + i * T));
    }
    float2 wc[stage_twiddle_count<M, E>() + 1];
    load_stage_twiddles_e<M, E, true>(t, tw, wc);
    bool late = false;
    for (int s = 0; s < S; ++s) {
        __syncthreads();  // every thread is done with the buffer that the next copy overwrites
        if (threadIdx.x == 0 && s + 1 < S) {
            ac::fence_proxy_async();
            fetch(s + 1, (s + 1) & 1);
        }
        if (!ac::mbar_wait(&full[s & 1], (s >> 1) & 1)) late = true;
        const float2* X = stage + (s & 1) * LZ * SP + li * SP;
        float2 v[E];
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int k = t + i * T;
            const float2 xk = X[k];
            const float2 xc = cconj((k == 0) ? make_float2(0.f, 0.f) : X[M - k]);
            const float2 a = cadd(xk, xc);
            const float2 c = cmul(WKS ? swk[k] : wk[i], csub(xk, xc));
            v[i] = make_float2(a.x - c.y, a.y + c.x);
        }
        fft_line_e_wc<M, E, true>(v, t, tw, sm, wc);
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < E; ++i) acc = fmaf(d2[i].x, v[i].x, fmaf(d2[i].y, v[i].y, acc));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) wdd[wid][s] = acc;
    }
    if (late) atomicOr(err, 4u);
    __syncthreads();
    if (threadIdx.x < S) {
        double tot = 0.0;
        for (int w = 0; w < NW; ++w) tot += (double)wdd[w][threadIdx.x];
        double* slot = dd_part + (size_t)threadIdx.x * (SLOTS * gridDim.x) + SLOTS * blockIdx.x;
        slot[0] = tot;
#pragma unroll
        for (int k = 1; k < SLOTS; ++k) slot[k] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// c2r along z of one filtered spectrum, written out as a real field (no
// contraction): out[line*N + 2j] = scale * Re z_j, out[line*N + 2j+1] = scale * Im z_j,
// with the same split of the half spectrum as I3.  Used to read a smoothed
// density back at the particles.
template <int N>
__global__ void __launch_bounds__(Cfg<N>::ZTHREADS) k_inv_z_c2r_store(const float2* __restrict__ work,
                                                                      float* __restrict__ out, float scale,
                                                                      const float2* __restrict__ tw) {
    using C = Cfg<N>;
    constexpr int M = C::MZ, T = C::TZ, LP = LinePad<M>::value, H = N / 2;
    extern __shared__ float2 smem[];
    const int t = threadIdx.x % T, li = threadIdx.x / T;
    const size_t line = (size_t)blockIdx.x * C::LZ + li;
    const SmemZLine<M> sm{{smem + li * LP}, li};
    const float2* X = work + line * H;
    float2 v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int k = t + i * T;
        const float2 xk = X[k];
        const float2 xc = cconj(k == 0 ? make_float2(0.f, 0.f) : X[M - k]);
        const float2 a = cadd(xk, xc);
        const float2 w = cconj(__ldg(tw + N + k));  // e^{+2 pi i k / N}
        const float2 c = cmul(w, csub(xk, xc));
        v[i] = make_float2(a.x - c.y, a.y + c.x);
    }
    fft_line<M, true>(v, t, tw, sm);
    float2* o = reinterpret_cast<float2*>(out + line * N);
#pragma unroll
    for (int i = 0; i < 8; ++i) o[t + i * T] = cscale(v[i], scale);
}

template <int N>
static cudaError_t smooth_impl(const float2* spec, float2* work, float* out, const WinBatch& wb, const Tables& tb,
                               cudaStream_t st, const Tracer& tr) {
    using C = Cfg<N>;
    cudaError_t e;
    if ((e = allow_smem(k_inv_x_window<N, false>, C::SMEM_STRIDED)) != cudaSuccess) return e;
    if ((e = allow_smem(k_strided<N, true>, C::SMEM_STRIDED)) != cudaSuccess) return e;
    if ((e = allow_smem(k_inv_z_c2r_store<N>, C::SMEM_Z)) != cudaSuccess) return e;
    const long long H = N / 2;
    tr(K_INV_X_WINDOW, 0, st);
    k_inv_x_window<N, false><<<dim3(H / C::W, N, 1), C::TS, C::SMEM_STRIDED, st>>>(spec, work, wb, tb);
    tr(K_INV_X_WINDOW, 1, st);
    tr(K_INV_Y, 0, st);
    k_strided<N, true><<<dim3(H / C::W, N, 1), C::TS, C::SMEM_STRIDED, st>>>(work, H, (long long)N * H, 0, 0, tb.tw);
    tr(K_INV_Y, 1, st);
    tr(K_INV_Z_STORE, 0, st);
    const float scale = 1.0f / ((float)N * (float)N * (float)N);
    k_inv_z_c2r_store<N><<<(N * N) / C::LZ, C::ZTHREADS, C::SMEM_Z, st>>>(work, out, scale, tb.tw);
    tr(K_INV_Z_STORE, 1, st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused I2 + I3 on a thread-block cluster.  The (y, k_z) plane of one x and one
// window (N x N/2 complex, 1 MiB at N = 512) is split over CL CTAs:
//   y phase : CTA c holds the k_z slab [c*KZ, (c+1)*KZ) for every y and runs the
//             inverse y FFTs (strided tile, as I2);
//   exchange: every element is written into the shared memory of the CTA that
//             owns its y line (distributed shared memory, one cluster barrier);
//   z phase : CTA c owns the y lines [c*YP, (c+1)*YP): complex-to-real along z
//             and the contraction with delta, whose slab stays in shared memory
//             for every window of the batch.
// Per window the plane is read from HBM once (4 B per cell) and never written.
namespace cg = cooperative_groups;

template <int N>
struct YZCfg {
    static constexpr int H = N / 2;
    static constexpr int CL = (N >= 512) ? 16 : (N == 256 ? 4 : 1);
    static constexpr int KZ = H / CL;                 // k_z columns per CTA (y phase)
    static constexpr int YP = N / CL;                 // y lines per CTA (z phase)
    static constexpr int THREADS = KZ * (N / 8);
    static_assert(THREADS == YP * (H / 8), "both phases use every thread");
    static constexpr int A_WORDS = SmemStrided<KZ>::words(N);
    static constexpr int LPB = LinePad<H>::value;
    static constexpr int B_WORDS = YP * LPB;
    static constexpr size_t SMEM = (size_t)(A_WORDS + B_WORDS + YP * H) * sizeof(float2);
};

template <int N>
__device__ __forceinline__ void yz_cluster_sync() {
    if constexpr (YZCfg<N>::CL > 1) cg::this_cluster().sync();
    else __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(YZCfg<N>::THREADS, 1)
    k_inv_yz_contract(const float2* __restrict__ work, int S, const float* __restrict__ delta,
                      const float2* __restrict__ tw, double* __restrict__ dd_part) {
    using C = YZCfg<N>;
    constexpr int H = N / 2, CL = C::CL, KZ = C::KZ, YP = C::YP, TY = N / 8, TZ = H / 8, LPB = C::LPB;
    constexpr int NW = (C::THREADS + 31) / 32;
    constexpr unsigned MASK = C::THREADS >= 32 ? 0xffffffffu : ((1u << C::THREADS) - 1u);
    extern __shared__ float4 smem_raw[];
    float2* bufA = reinterpret_cast<float2*>(smem_raw);
    float2* bufB = bufA + C::A_WORDS;
    float2* dsl = bufB + C::B_WORDS;  // delta slab, pairs (2j, 2j+1): [YP][H]
    __shared__ float wdd[NW][MAX_BATCH];
    const int x = blockIdx.y;
    int c = 0;
    if constexpr (CL > 1) c = (int)cg::this_cluster().block_rank();
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int col = tid % KZ, ty = tid / KZ;          // y phase
    const int tz = tid % TZ, yl = tid / TZ;           // z phase
    const int kz0 = c * KZ;
    const float2* dsrc = reinterpret_cast<const float2*>(delta + ((size_t)x * N + (size_t)c * YP) * N);
    for (int e = tid; e < YP * H; e += C::THREADS) dsl[e] = dsrc[e];
    yz_cluster_sync<N>();  // every CTA of the cluster runs before any remote access
    for (int s = 0; s < S; ++s) {
        const float2* src = work + (size_t)s * N * N * H + (size_t)x * N * H + kz0 + col;
        float2 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = src[(size_t)(ty + i * TY) * H];
        fft_line<N, true>(v, ty, tw, SmemStrided<KZ>{bufA, col});
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int y = ty + i * TY;
            float2* rb = bufB;
            if constexpr (CL > 1) rb = cg::this_cluster().map_shared_rank(bufB, y / YP);
            rb[(y % YP) * LPB + SmemLine<H>::at(kz0 + col)] = v[i];
        }
        yz_cluster_sync<N>();  // the transposed plane is complete in every CTA
        const SmemLine<H> sm{bufB + yl * LPB};
        float2 w[8], xm[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = tz + i * TZ;
            w[i] = sm.ld(k);
            xm[i] = (k == 0) ? make_float2(0.f, 0.f) : sm.ld(H - k);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = tz + i * TZ;
            const float2 xc = cconj(xm[i]);
            const float2 a = cadd(w[i], xc);
            const float2 wk = cconj(__ldg(tw + N + k));  // e^{+2 pi i k / N}
            const float2 cc = cmul(wk, csub(w[i], xc));
            w[i] = make_float2(a.x - cc.y, a.y + cc.x);
        }
        fft_line<H, true>(w, tz, tw, sm);
        float acc = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float2 d = dsl[yl * H + tz + i * TZ];
            acc = fmaf(d.x, w[i].x, fmaf(d.y, w[i].y, acc));
        }
#pragma unroll
        for (int o = (C::THREADS >= 32 ? 16 : C::THREADS / 2); o > 0; o >>= 1) acc += __shfl_xor_sync(MASK, acc, o);
        if (lane == 0) wdd[wid][s] = acc;
        yz_cluster_sync<N>();  // every CTA finished reading its plane slice before the next scatter
    }
    __syncthreads();
    if (tid < S) {
        double tot = 0.0;
        for (int q = 0; q < NW; ++q) tot += (double)wdd[q][tid];
        const size_t nblk = (size_t)gridDim.y * CL;
        dd_part[(size_t)tid * nblk + (size_t)x * CL + c] = tot;
    }
}

// Whether the fused y-z pass runs: only when HERMES_YZ_FUSED=1 (opt-in: with one
// 1024-thread CTA per SM and two cluster barriers per window it is latency-bound
// and slower than the separate y and z passes on B300), N <= 512, and a cluster
// of CL CTAs with SMEM bytes each fits the device.
template <int N>
static bool yz_fused_ok() {
    if constexpr (N > 512) {
        return false;
    } else {
        const char* env = getenv("HERMES_YZ_FUSED");
        if (!env || env[0] != '1') return false;
        static int state = -1;  // per N: -1 unknown, 0 no, 1 yes
        if (state >= 0) return state == 1;
        using C = YZCfg<N>;
        state = 0;
        if (cudaFuncSetAttribute(k_inv_yz_contract<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM) !=
            cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (C::CL > 8 &&
            cudaFuncSetAttribute(k_inv_yz_contract<N>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (C::CL > 1) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = C::CL;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(C::CL, N, 1);
            cfg.blockDim = dim3(C::THREADS, 1, 1);
            cfg.dynamicSmemBytes = C::SMEM;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, k_inv_yz_contract<N>, &cfg) != cudaSuccess ||
                nclusters < 1) {
                cudaGetLastError();
                return false;
            }
        }
        state = 1;
        return true;
    }
}

template <int N>
static cudaError_t launch_yz(const float2* work, int S, const float* delta, const float2* tw, double* dd_part,
                             cudaStream_t st) {
    using C = YZCfg<N>;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C::CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C::CL, N, 1);
    cfg.blockDim = dim3(C::THREADS, 1, 1);
    cfg.dynamicSmemBytes = C::SMEM;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_inv_yz_contract<N>, work, S, delta, tw, dd_part);
}

// ---------------------------------------------------------------------------
// host launchers

template <int N>
static cudaError_t forward_impl(float* grid, float2* spec, const double* scal, int convert, const Tables& tb,
                                cudaStream_t st, const Tracer& tr, int ncat, int keep_dc = 0) {
    using C = Cfg<N>;
    cudaError_t e;
    if ((e = allow_smem(k_fwd_z_r2c<N>, C::SMEM_Z)) != cudaSuccess) return e;
    if ((e = allow_smem(k_strided<N, false>, C::SMEM_STRIDED)) != cudaSuccess) return e;
    tr(K_FWD_Z_R2C, 0, st);
    k_fwd_z_r2c<N><<<dim3((N * N) / C::LZ, ncat), C::ZTHREADS, C::SMEM_Z, st>>>(grid, spec, scal, convert, tb.tw);
    tr(K_FWD_Z_R2C, 1, st);
    const long long H = N / 2;
    const long long cat_stride = (long long)N * N * H;  // one spectrum per catalogue (blockIdx.z)
    dim3 g(H / C::W, N, ncat);
    // along y: pos stride H, blockIdx.y = x
    tr(K_FWD_Y, 0, st);
    k_strided<N, false><<<g, C::TS, C::SMEM_STRIDED, st>>>(spec, H, (long long)N * H, cat_stride, 0, tb.tw);
    tr(K_FWD_Y, 1, st);
    // along x: pos stride N*H, blockIdx.y = y, delta^(0) := 0
    tr(K_FWD_X, 0, st);
    k_strided<N, false><<<g, C::TS, C::SMEM_STRIDED, st>>>(spec, (long long)N * H, H, cat_stride, keep_dc ? 0 : 1,
                                                            tb.tw);
    tr(K_FWD_X, 1, st);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Variants of the tuned FFT passes and the autotuner that picks one per pass and grid
// size.  A variant fixes the values per thread E (the radix of the FFT stages: radix 8
// throughout for E = 8, radix 16 or 32 for E = 16, 32), the tile width W, the blocks per
// SM it is compiled for (minb, 0: not fixed) and a kind:
//   pass 0, the inverse y pass (I2): 0 the radix-8 pass (k_strided_pf up to 512^3,
//           k_strided above), 1 one tile per block (k_strided_e; k_inv_y_e, the strides
//           fixed at compile time, for the 16-column tiles), 2 k_strided_pf_e
//           (persistent);
//   pass 1, the window pass (I1): 0 one window at a time (k_inv_x_window, shared table
//           when it fits), 1 k_inv_x_window_pair (two windows in flight per thread),
//           2 k_inv_x_window_mirror (the k_y and N - k_y lines together, one table read
//           for both), 3 the same reading one radial factor per element and window
//           instead of four windows' factors at once (24 registers fewer), 4 (512^3) the
//           same storing both lines of a column in one 16-byte store, in the paired order
//           (whole 128-byte lines); the y pass then reads that order (its variants 4 and
//           5 have a form for it; with another y variant, variant 3 runs in its place),
//           5 (512^3) the paired order written by tiled bulk stores (TMA) of a shared stage;
//   pass 2, the c2r + contraction pass (I3): 0 radix 8 (k_inv_z_c2r_contract),
//           1 k_inv_z_c2r_contract_e16 (16 values per thread, 128-thread blocks), 2 the same
//           with its split twiddles in a table shared by the block (no spills);
//   pass 3, the zeta_l y pass: 0 radix 8 (k_strided), 1 k_strided_e (k_inv_y_e for the
//           16-column tiles);
//   passes 4, 5, the zeta_l x pass for complex / packed m = 0 fields: 0 one line set at
//           a time (k_zeta_x), 2 the k_y and N - k_y lines together (k_zeta_x_mirror), 3 the
//           same reading each field's radial factors when used (no spills), 4 (512^3) the
//           same in the paired order, read by the zeta_l y pass's variants 3 and 4 (with
//           another y variant, kind 3 runs in its place).
// The first call of a grid size that runs a pass on a stream that is not being captured
// into a graph times every variant on that call's own buffers (the y passes before the
// passes that write their buffers, the others on the first catalogue), one warm-up and two
// timed launches each, and keeps the fastest for the process and device;
// hermes_fft_set_variant fixes one instead.  The choice is made for the shape of that
// first call (windows per launch, orders, bins) and kept for later calls of other shapes.

static int sm_count() {
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

struct PassVariant {
    int kind, E, W, minb;
};
constexpr int kMaxVariants = 8;
static int pass_variants(int N, int pass, PassVariant* out) {
    auto put = [&](std::initializer_list<PassVariant> l) {
        int k = 0;
        for (const PassVariant& v : l) out[k++] = v;
        return k;
    };
    if (pass == 0) {
        switch (N) {
            case 16: return put({{0, 8, Cfg<16>::W, 2}});
            case 32: return put({{0, 8, Cfg<32>::W, 2}});
            case 64: return put({{0, 8, Cfg<64>::W, 2}});
            case 128: return put({{0, 8, Cfg<128>::W, 2}, {1, 16, 8, 0}});
            case 256: return put({{0, 8, Cfg<256>::W, 2}, {1, 16, 8, 0}, {2, 16, 8, 3}, {1, 32, 8, 0},
                                  {1, 16, 16, 2}, {1, 32, 16, 4}});
            case 512: return put({{0, 8, Cfg<512>::W, 2}, {2, 32, 8, 2}, {1, 32, 8, 0}, {1, 16, 8, 0},
                                  {1, 32, 16, 1}, {1, 32, 16, 2}});
            case 1024: return put({{0, 8, Cfg<1024>::W, 0}, {1, 32, 8, 0}, {1, 16, 8, 0}});
        }
    } else if (pass == 2) {
        switch (N) {
            case 256: return put({{0, 8, 1, 3}, {1, 16, 1, 4}, {1, 16, 1, 3}, {1, 16, 1, 2}, {2, 16, 1, 4}});
            case 512: return put({{0, 8, 1, 3}, {1, 16, 1, 4}, {1, 16, 1, 3}, {1, 16, 1, 2}, {2, 16, 1, 4}});
            case 16: case 32: case 64: case 128: case 1024: return put({{0, 8, 1, 3}});
        }
    } else if (pass == 4 || pass == 5) {  // the zeta_l x pass: complex fields / packed m = 0 fields
        switch (N) {
            case 16: return put({{0, 8, Cfg<16>::W, 1}});
            case 32: return put({{0, 8, Cfg<32>::W, 1}});
            case 64: return put({{0, 8, Cfg<64>::W, 1}});
            case 128: return put({{0, 8, Cfg<128>::W, 1}});
            case 256: return put({{0, 8, Cfg<256>::W, 1}, {2, 8, Cfg<256>::W, 1}, {3, 8, Cfg<256>::W, 1}});
            case 512: return put({{0, 8, Cfg<512>::W, 1}, {2, 8, Cfg<512>::W, 1}, {3, 8, Cfg<512>::W, 1},
                                  {4, 8, Cfg<512>::W, 1}});
            case 1024: return put({{0, 8, Cfg<1024>::W, 1}});
        }
    } else if (pass == 3) {
        switch (N) {
            case 16: return put({{0, 8, Cfg<16>::W, 0}});
            case 32: return put({{0, 8, Cfg<32>::W, 0}});
            case 64: return put({{0, 8, Cfg<64>::W, 0}});
            case 128: return put({{0, 8, Cfg<128>::W, 0}});
            case 256: return put({{0, 8, Cfg<256>::W, 0}, {1, 16, 8, 0}, {1, 32, 8, 0}, {1, 16, 16, 2},
                                  {1, 32, 16, 4}});
            case 512: return put({{0, 8, Cfg<512>::W, 0}, {1, 32, 8, 0}, {1, 16, 8, 0}, {1, 32, 16, 1},
                                  {1, 32, 16, 2}});
            case 1024: return put({{0, 8, Cfg<1024>::W, 0}});
        }
    } else if (pass == 1) {
        switch (N) {
            case 16: return put({{0, 8, Cfg<16>::W, 1}});
            case 32: return put({{0, 8, Cfg<32>::W, 1}});
            case 64: return put({{0, 8, Cfg<64>::W, 1}});
            case 128: return put({{0, 8, Cfg<128>::W, 1}});
            case 256: return put({{0, 8, Cfg<256>::W, 1}, {1, 8, Cfg<256>::W, 1}, {2, 8, Cfg<256>::W, 1},
                                  {3, 8, Cfg<256>::W, 1}});
            case 512: return put({{0, 8, Cfg<512>::W, 1}, {1, 8, Cfg<512>::W, 1}, {2, 8, Cfg<512>::W, 1},
                                  {3, 8, Cfg<512>::W, 1}, {4, 8, Cfg<512>::W, 1}, {5, 8, Cfg<512>::W, 1}});
            case 1024: return put({{0, 8, Cfg<1024>::W, 1}});
        }
    }
    return 0;
}

// Tiles (column chunk, x, window) of nwin consecutive windows of work.
template <int N>
static cudaError_t run_y_r8(float2* work, int nwin, const float2* tw, cudaStream_t st) {
    using C = Cfg<N>;
    constexpr long long H = N / 2;
    cudaError_t e;
    const int nxt = (int)(H / C::W);
    const long long ntiles = (long long)nxt * N * nwin;
    if constexpr (N <= 512) {  // two 512-thread blocks per SM at 64 registers
        if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
        if ((e = allow_smem(k_strided_pf<N, true>, C::SMEM_STRIDED)) != cudaSuccess) return e;
        const int nblk = (int)std::min<long long>(ntiles, 2LL * sm_count());
        k_strided_pf<N, true><<<nblk, C::TS, C::SMEM_STRIDED, st>>>(work, (int)H, (int)(N * H), (long long)N * N * H,
                                                                    nxt, N, (int)ntiles, tw);
    } else {
        if ((e = allow_smem(k_strided<N, true>, C::SMEM_STRIDED)) != cudaSuccess) return e;
        dim3 g2(nxt, N, nwin);
        k_strided<N, true><<<g2, C::TS, C::SMEM_STRIDED, st>>>(work, H, (long long)N * H, (long long)N * N * H, 0, tw);
    }
    return cudaGetLastError();
}
template <int N, int E, int W, int SH, int P>
static cudaError_t run_y_plain(float2* work, int nwin, const float2* tw, cudaStream_t st) {
    constexpr int H = N / 2, TS = (N / E) * W;
    constexpr size_t smem = (size_t)SmemStridedSk<W, SH, P>::words(N) * sizeof(float2);
    cudaError_t e;
    if ((e = allow_smem(k_strided_e<N, E, W, SH, P>, smem)) != cudaSuccess) return e;
    k_strided_e<N, E, W, SH, P><<<dim3(H / W, N, nwin), TS, smem, st>>>(work, H, N * H, (long long)N * N * H, tw);
    return cudaGetLastError();
}
template <int N, int Z, int E, int W, int SH, int P, int MINB, bool PAIRED = false>
static cudaError_t run_y_ct(float2* data, int nf, const float2* tw, cudaStream_t st) {
    constexpr int TS = (N / E) * W;
    constexpr size_t smem = (size_t)SmemStridedSk<W, SH, P>::words(N) * sizeof(float2);
    cudaError_t e;
    if ((e = allow_smem(k_inv_y_e<N, Z, E, W, SH, P, MINB, PAIRED>, smem)) != cudaSuccess) return e;
    k_inv_y_e<N, Z, E, W, SH, P, MINB, PAIRED><<<dim3(Z / W, N, nf), TS, smem, st>>>(data, tw);
    return cudaGetLastError();
}
template <int N, int E, int W, int SH, int P, int MINB>
static cudaError_t run_y_pf(float2* work, int nwin, const float2* tw, cudaStream_t st) {
    constexpr int H = N / 2, TS = (N / E) * W;
    constexpr size_t smem = (size_t)SmemStridedSk<W, SH, P>::words(N) * sizeof(float2);
    const int nxt = H / W;
    const long long ntiles = (long long)nxt * N * nwin;
    if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = allow_smem(k_strided_pf_e<N, E, W, SH, P, MINB>, smem)) != cudaSuccess) return e;
    const int nblk = (int)std::min<long long>(ntiles, (long long)MINB * sm_count());
    k_strided_pf_e<N, E, W, SH, P, MINB><<<nblk, TS, smem, st>>>(work, H, N * H, (long long)N * N * H, nxt, N,
                                                                  (int)ntiles, tw);
    return cudaGetLastError();
}
// The skews (SH, P) below give the fewest shared-memory wavefronts for each shape.
// paired: the input is in the paired order of the window pass (variants 4 and 5 at 512^3).
template <int N>
static cudaError_t launch_inv_y(int var, float2* work, int nwin, const float2* tw, cudaStream_t st,
                                bool paired = false) {
    if constexpr (N == 512) {
        if (paired) {
            if (var == 4) return run_y_ct<512, 256, 32, 16, 3, 0, 1, true>(work, nwin, tw, st);
            if (var == 5) return run_y_ct<512, 256, 32, 16, 3, 0, 2, true>(work, nwin, tw, st);
            return cudaErrorInvalidValue;
        }
    }
    if (paired) return cudaErrorInvalidValue;
    if constexpr (N == 128) {
        if (var == 1) return run_y_plain<128, 16, 8, 2, 4>(work, nwin, tw, st);
    } else if constexpr (N == 256) {
        if (var == 1) return run_y_plain<256, 16, 8, 2, 2>(work, nwin, tw, st);
        if (var == 2) return run_y_pf<256, 16, 8, 2, 2, 3>(work, nwin, tw, st);
        if (var == 3) return run_y_plain<256, 32, 8, 2, 4>(work, nwin, tw, st);
        if (var == 4) return run_y_ct<256, 128, 16, 16, 3, 0, 2>(work, nwin, tw, st);
        if (var == 5) return run_y_ct<256, 128, 32, 16, 3, 0, 4>(work, nwin, tw, st);
    } else if constexpr (N == 512) {
        if (var == 1) return run_y_pf<512, 32, 8, 2, 2, 2>(work, nwin, tw, st);
        if (var == 2) return run_y_plain<512, 32, 8, 2, 2>(work, nwin, tw, st);
        if (var == 3) return run_y_plain<512, 16, 8, 2, 1>(work, nwin, tw, st);
        // strides fixed at compile time; 16-column tiles read and write whole 128-byte lines
        // (no skew needed at that width)
        if (var == 4) return run_y_ct<512, 256, 32, 16, 3, 0, 1>(work, nwin, tw, st);
        if (var == 5) return run_y_ct<512, 256, 32, 16, 3, 0, 2>(work, nwin, tw, st);
    } else if constexpr (N == 1024) {
        if (var == 1) return run_y_plain<1024, 32, 8, 2, 1>(work, nwin, tw, st);
        if (var == 2) return run_y_plain<1024, 16, 8, 2, 8>(work, nwin, tw, st);
    }
    return run_y_r8<N>(work, nwin, tw, st);
}

// The window pass: tiles of W k_z columns at one k_y (grid (H / W, N, ncat)).
template <int N>
static cudaError_t run_x_r8(const float2* spec, float2* work, const WinBatch& wb, const Tables& tb, int ncat,
                            cudaStream_t st) {
    using C = Cfg<N>;
    cudaError_t e;
    // radial factors staged in shared memory when they fit next to the FFT tile
    const size_t stab_bytes = C::SMEM_STRIDED + (size_t)(N / 2) * C::W * stab_row_stride(wb.S) * sizeof(float);
    const bool use_stab = stab_bytes <= kMaxDynSmem && stab_x_enabled();
    dim3 g1((N / 2) / C::W, N, ncat);
    if (use_stab) {
        if ((e = allow_smem(k_inv_x_window<N, true>, stab_bytes)) != cudaSuccess) return e;
        k_inv_x_window<N, true><<<g1, C::TS, stab_bytes, st>>>(spec, work, wb, tb);
    } else {
        if ((e = allow_smem(k_inv_x_window<N, false>, C::SMEM_STRIDED)) != cudaSuccess) return e;
        k_inv_x_window<N, false><<<g1, C::TS, C::SMEM_STRIDED, st>>>(spec, work, wb, tb);
    }
    return cudaGetLastError();
}
template <int N>
static cudaError_t run_x_pair(const float2* spec, float2* work, const WinBatch& wb, const Tables& tb, int ncat,
                              cudaStream_t st) {
    using C = Cfg<N>;
    const size_t bytes = 2 * C::SMEM_STRIDED + (size_t)(N / 2) * C::W * pair_row_floats(wb.S) * sizeof(float);
    if (wb.S > 16 || bytes > kMaxDynSmem) return run_x_r8<N>(spec, work, wb, tb, ncat, st);
    cudaError_t e;
    if ((e = allow_smem(k_inv_x_window_pair<N>, bytes)) != cudaSuccess) return e;
    k_inv_x_window_pair<N><<<dim3((N / 2) / C::W, N, ncat), C::TS, bytes, st>>>(spec, work, wb, tb);
    return cudaGetLastError();
}
template <int N>
static bool mirror_fits(const WinBatch& wb) {
    using C = Cfg<N>;
    const size_t bytes = 2 * C::SMEM_STRIDED + (size_t)(N / 2) * C::W * pair_row_floats(wb.S) * sizeof(float);
    return wb.S <= 16 && bytes <= kMaxDynSmem;
}
// The tensor map of the paired-order stores of k_inv_x_window_mirror<512, ..., TMA>: the
// work buffer of nwin windows as float32 [nwin * N][N][N] (k_z fastest, as real and
// imaginary parts), boxes of 32 floats (one 16-column group) x 1 line x N/2 x planes.
// false when the driver's encoder is unavailable or refuses the map.
static bool encode_paired_store_map(CUtensorMap* map, float2* work, int N, long long nwin) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode || (reinterpret_cast<uintptr_t>(work) & 15) != 0 || nwin * N > 0x7fffffffLL) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)(nwin * N)};
    const cuuint64_t strides[2] = {(cuuint64_t)N * sizeof(float), (cuuint64_t)N * N * sizeof(float)};
    const cuuint32_t box[3] = {32, 1, (cuuint32_t)(N / 2)};
    const cuuint32_t estr[3] = {1, 1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, work, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The paired order never falls back to the plain one: the y pass that follows reads it.
// TMA: the paired order by tiled bulk stores (512^3); the threads' own stores when the
// tensor map cannot be made.
template <int N, bool ONE, bool PAIRED = false, bool TMA = false>
static cudaError_t run_x_mirror(const float2* spec, float2* work, const WinBatch& wb, const Tables& tb, int ncat,
                                cudaStream_t st) {
    using C = Cfg<N>;
    const size_t bytes = 2 * C::SMEM_STRIDED + (size_t)(N / 2) * C::W * pair_row_floats(wb.S) * sizeof(float);
    if (!mirror_fits<N>(wb)) return PAIRED ? cudaErrorInvalidValue : run_x_r8<N>(spec, work, wb, tb, ncat, st);
    alignas(64) CUtensorMap map{};
    if constexpr (TMA) {
        if (!encode_paired_store_map(&map, work, N, (long long)wb.S * ncat))
            return run_x_mirror<N, ONE, true, false>(spec, work, wb, tb, ncat, st);
    }
    cudaError_t e;
    if ((e = allow_smem(k_inv_x_window_mirror<N, ONE, PAIRED, TMA>, bytes)) != cudaSuccess) return e;
    k_inv_x_window_mirror<N, ONE, PAIRED, TMA><<<dim3((N / 2) / C::W, PAIRED ? N / 2 : N / 2 + 1, ncat), C::TS,
                                                 bytes, st>>>(spec, work, wb, tb, map);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_inv_x(int var, const float2* spec, float2* work, const WinBatch& wb, const Tables& tb,
                                int ncat, cudaStream_t st) {
    if constexpr (N == 256 || N == 512) {
        switch (var) {
            case 1: return run_x_pair<N>(spec, work, wb, tb, ncat, st);
            case 2: return run_x_mirror<N, false>(spec, work, wb, tb, ncat, st);
            case 3: return run_x_mirror<N, true>(spec, work, wb, tb, ncat, st);
        }
    }
    if constexpr (N == 512) {
        if (var == 4) return run_x_mirror<N, true, true>(spec, work, wb, tb, ncat, st);
        if (var == 5) return run_x_mirror<N, true, true, true>(spec, work, wb, tb, ncat, st);
    }
    return run_x_r8<N>(spec, work, wb, tb, ncat, st);
}
// Whether the window pass variant writes the paired order, and whether the y pass
// variant has a form that reads it.
template <int N>
static bool x_writes_paired(int xvar) {
    return N == 512 && (xvar == 4 || xvar == 5);
}
template <int N>
static bool y_reads_paired(int yvar) {
    return N == 512 && (yvar == 4 || yvar == 5);
}

// The last inverse pass (c2r along z and the contraction): delta of the first catalogue
// of the launch at delta, partials [ncat][S][z blocks of the radix-8 form].
template <int N, int THREADS, int MINB, bool WKS = false>
static cudaError_t run_z_e16(const float2* work, int S, const float* delta, const float2* tw, double* dd_part,
                             unsigned* err, int ncat, cudaStream_t st) {
    using C = Z16Cfg<N, THREADS>;
    cudaError_t e;
    if ((e = allow_smem(k_inv_z_c2r_contract_e16<N, THREADS, MINB, WKS>, C::SMEM)) != cudaSuccess) return e;
    k_inv_z_c2r_contract_e16<N, THREADS, MINB, WKS><<<dim3((N * N) / C::LZ, ncat), THREADS, C::SMEM, st>>>(
        work, S, delta, tw, dd_part, err);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_inv_z(int var, const float2* work, int S, const float* delta, const float2* tw,
                                double* dd_part, unsigned* err, int ncat, cudaStream_t st) {
    if constexpr (N == 256 || N == 512) {  // at 1024^3 (512-point lines) radix 8 measured as fast
        if (var == 1) return run_z_e16<N, 128, 4>(work, S, delta, tw, dd_part, err, ncat, st);
        if (var == 2) return run_z_e16<N, 128, 3>(work, S, delta, tw, dd_part, err, ncat, st);
        if (var == 3) return run_z_e16<N, 128, 2>(work, S, delta, tw, dd_part, err, ncat, st);
        if (var == 4) return run_z_e16<N, 128, 4, true>(work, S, delta, tw, dd_part, err, ncat, st);
    }
    using C = Cfg<N>;
    k_inv_z_c2r_contract<N><<<dim3((N * N) / C::LZ, ncat), C::ZTHREADS, C::SMEM_Z3, st>>>(work, S, delta, tw,
                                                                                        dd_part, err);
    return cudaGetLastError();
}

// The inverse y transform of the zeta_l harmonic fields (pass 3): nf fields of N^3
// complex values, [f][x][y][z]; tiles of W adjacent z columns at one (x, f).  Variant
// 0 is the radix-8 strided pass (the tile of the zeta y pass: Cfg<N>::W columns).
template <int N, int E, int W, int SH, int P>
static cudaError_t run_zeta_y_e(float2* fields, int nf, const float2* tw, cudaStream_t st) {
    constexpr int TS = (N / E) * W;
    constexpr size_t smem = (size_t)SmemStridedSk<W, SH, P>::words(N) * sizeof(float2);
    cudaError_t e;
    if ((e = allow_smem(k_strided_e<N, E, W, SH, P>, smem)) != cudaSuccess) return e;
    k_strided_e<N, E, W, SH, P><<<dim3(N / W, N, nf), TS, smem, st>>>(fields, N, N * N, (long long)N * N * N, tw);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_zeta_y_var(int var, float2* fields, int nf, const float2* tw, cudaStream_t st,
                                     bool paired = false) {
    if constexpr (N == 512) {
        if (paired) {  // the fields in the paired order of the x pass (its variant 3)
            if (var == 3) return run_y_ct<512, 512, 32, 16, 3, 0, 1, true>(fields, nf, tw, st);
            if (var == 4) return run_y_ct<512, 512, 32, 16, 3, 0, 2, true>(fields, nf, tw, st);
            return cudaErrorInvalidValue;
        }
    }
    if (paired) return cudaErrorInvalidValue;
    if constexpr (N == 256) {
        if (var == 1) return run_zeta_y_e<256, 16, 8, 2, 2>(fields, nf, tw, st);
        if (var == 2) return run_zeta_y_e<256, 32, 8, 2, 4>(fields, nf, tw, st);
        if (var == 3) return run_y_ct<256, 256, 16, 16, 3, 0, 2>(fields, nf, tw, st);
        if (var == 4) return run_y_ct<256, 256, 32, 16, 3, 0, 4>(fields, nf, tw, st);
    } else if constexpr (N == 512) {
        if (var == 1) return run_zeta_y_e<512, 32, 8, 2, 2>(fields, nf, tw, st);
        if (var == 2) return run_zeta_y_e<512, 16, 8, 2, 1>(fields, nf, tw, st);
        if (var == 3) return run_y_ct<512, 512, 32, 16, 3, 0, 1>(fields, nf, tw, st);
        if (var == 4) return run_y_ct<512, 512, 32, 16, 3, 0, 2>(fields, nf, tw, st);
    }
    using C = Cfg<N>;
    cudaError_t e;
    if ((e = allow_smem(k_strided<N, true>, C::SMEM_STRIDED)) != cudaSuccess) return e;
    k_strided<N, true><<<dim3(N / C::W, N, nf), C::TS, C::SMEM_STRIDED, st>>>(fields, N, (long long)N * N,
                                                                            (long long)N * N * N, 0, tw);
    return cudaGetLastError();
}

struct Tune {
    int forced = -1, chosen = -1;
    double ms[kMaxVariants];
    Tune() {
        for (double& m : ms) m = -1.0;
    }
};
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int>, Tune> g_tune;  // (device, N, pass)

static std::tuple<int, int, int> tune_key(int N, int pass) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
    return {dev, N, pass};
}

// The variant of this call for (N, pass): the forced one, else the tuned one, else
// (timing trial(v), one launch of variant v on the call's buffers, when st is not
// capturing) the fastest; variant 0 while capturing before any tuning.
template <class F>
static int pick_variant(int N, int pass, cudaStream_t st, F&& trial) {
    PassVariant vs[kMaxVariants];
    const int nvar = pass_variants(N, pass, vs);
    if (nvar <= 1) return 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    Tune& en = g_tune[tune_key(N, pass)];
    if (en.forced >= 0) return en.forced;
    if (en.chosen >= 0) return en.chosen;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return 0;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return 0;
    }
    int best = 0;
    double best_ms = 1e300;
    for (int v = 0; v < nvar; ++v) {
        en.ms[v] = -1.0;
        if (trial(v) != cudaSuccess) {  // warm-up
            cudaGetLastError();
            continue;
        }
        float ms = 0.f;
        if (cudaEventRecord(e0, st) != cudaSuccess || trial(v) != cudaSuccess || trial(v) != cudaSuccess ||
            cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        en.ms[v] = ms / 2.0;
        if (en.ms[v] < best_ms) best_ms = en.ms[v], best = v;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    en.chosen = best;
    return best;
}

template <int N>
static int zeta_y_pick(float2* fields, int nf, const float2* tw, cudaStream_t st) {
    // trials transform one field in place; the x pass rewrites every field afterwards
    return pick_variant(N, 3, st, [&](int v) { return launch_zeta_y_var<N>(v, fields, std::min(nf, 1), tw, st); });
}
int zeta_y_variant(int N, float2* fields, int nf, const float2* tw, cudaStream_t st) {
    if (nf < 1) return 0;
#define F(n) zeta_y_pick<n>(fields, nf, tw, st)
    switch (N) {
        case 16: return F(16);
        case 32: return F(32);
        case 64: return F(64);
        case 128: return F(128);
        case 256: return F(256);
        case 512: return F(512);
        case 1024: return F(1024);
    }
#undef F
    return 0;
}
bool zeta_y_reads_paired(int N, int var) { return N == 512 && (var == 3 || var == 4); }
cudaError_t launch_zeta_y(int N, int var, float2* fields, int nf, const float2* tw, cudaStream_t st, bool paired) {
    switch (N) {
        case 16: return launch_zeta_y_var<16>(var, fields, nf, tw, st, paired);
        case 32: return launch_zeta_y_var<32>(var, fields, nf, tw, st, paired);
        case 64: return launch_zeta_y_var<64>(var, fields, nf, tw, st, paired);
        case 128: return launch_zeta_y_var<128>(var, fields, nf, tw, st, paired);
        case 256: return launch_zeta_y_var<256>(var, fields, nf, tw, st, paired);
        case 512: return launch_zeta_y_var<512>(var, fields, nf, tw, st, paired);
        case 1024: return launch_zeta_y_var<1024>(var, fields, nf, tw, st, paired);
    }
    return cudaErrorInvalidValue;
}

int tuned_variant(int N, int pass, cudaStream_t st, cudaError_t (*trial)(int v, void* arg), void* arg) {
    return pick_variant(N, pass, st, [&](int v) { return trial(v, arg); });
}

int fft_variants(int N, int pass, int* desc, double* ms, int cap, int* chosen, int* forced) {
    PassVariant vs[kMaxVariants];
    const int n = pass_variants(N, pass, vs);
    if (n == 0) return -1;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const auto it = g_tune.find(tune_key(N, pass));
    for (int i = 0; i < std::min(n, cap); ++i) {
        if (desc) {
            desc[4 * i] = vs[i].kind;
            desc[4 * i + 1] = vs[i].E;
            desc[4 * i + 2] = vs[i].W;
            desc[4 * i + 3] = vs[i].minb;
        }
        if (ms) ms[i] = it == g_tune.end() ? -1.0 : it->second.ms[i];
    }
    if (chosen) *chosen = it == g_tune.end() ? -1 : it->second.chosen;
    if (forced) *forced = it == g_tune.end() ? -1 : it->second.forced;
    return n;
}

int fft_set_variant(int N, int pass, int variant) {
    PassVariant vs[kMaxVariants];
    const int n = pass_variants(N, pass, vs);
    if (n == 0 || variant < -1 || variant >= n) return -1;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    Tune& en = g_tune[tune_key(N, pass)];
    en.forced = variant;
    if (variant < 0) {  // back to autotuning: the next uncaptured call times the variants again
        en.chosen = -1;
        for (double& m : en.ms) m = -1.0;
    }
    return 0;
}

template <int N>
static cudaError_t inverse_impl(const float2* spec, float2* work, const float* delta, const WinBatch& wb,
                                const Tables& tb, double* dd_part, unsigned* err, cudaStream_t st, const Tracer& tr,
                                int ncat) {
    using C = Cfg<N>;
    cudaError_t e;
    if ((e = allow_smem(k_inv_z_c2r_contract<N>, C::SMEM_Z3)) != cudaSuccess) return e;
    // the pass variants, tuned on the first uncaptured call of this grid size: the y
    // pass on this call's work buffer before the window pass writes it (about 1 GiB
    // of it), the window pass on the first catalogue
    const bool yz = ncat == 1 && yz_fused_ok<N>();
    const size_t win_bytes = (size_t)N * N * (N / 2) * sizeof(float2);
    const int nwin_trial = (int)std::max<size_t>(1, std::min<size_t>((size_t)wb.S * ncat, ((size_t)1 << 30) / win_bytes));
    const int yvar = yz ? 0 : pick_variant(N, 0, st, [&](int v) { return launch_inv_y<N>(v, work, nwin_trial, tb.tw, st); });
    const int xvar = pick_variant(N, 1, st, [&](int v) { return launch_inv_x<N>(v, spec, work, wb, tb, 1, st); });
    // (the trials of the last pass read the work buffer as it is and write partials the real launch overwrites)
    const int zvar = yz ? 0 : pick_variant(N, 2, st, [&](int v) {
        return launch_inv_z<N>(v, work, wb.S, delta, tb.tw, dd_part, err, 1, st);
    });
    // the paired order of the window pass needs a y pass that reads it; otherwise the same
    // window pass runs with plain stores
    const bool paired = x_writes_paired<N>(xvar) && !yz && y_reads_paired<N>(yvar) && mirror_fits<N>(wb);
    const int xrun = x_writes_paired<N>(xvar) && !paired ? 3 : xvar;
    tr(K_INV_X_WINDOW, 0, st);
    if ((e = launch_inv_x<N>(xrun, spec, work, wb, tb, ncat, st)) != cudaSuccess) return e;
    tr(K_INV_X_WINDOW, 1, st);
    if constexpr (N <= 512) {
        if (yz) {
            tr(K_INV_YZ_CONTRACT, 0, st);
            e = launch_yz<N>(work, wb.S, delta, tb.tw, dd_part, st);
            tr(K_INV_YZ_CONTRACT, 1, st);
            return e != cudaSuccess ? e : cudaGetLastError();
        }
    }
    // windows of all catalogues are consecutive in work: tiles (column chunk, x, window)
    tr(K_INV_Y, 0, st);
    if ((e = launch_inv_y<N>(yvar, work, wb.S * ncat, tb.tw, st, paired)) != cudaSuccess) return e;
    tr(K_INV_Y, 1, st);
    tr(K_INV_Z_C2R_CONTRACT, 0, st);
    if ((e = launch_inv_z<N>(zvar, work, wb.S, delta, tb.tw, dd_part, err, ncat, st)) != cudaSuccess) return e;
    tr(K_INV_Z_C2R_CONTRACT, 1, st);
    return cudaGetLastError();
}

#define HERMES_DISPATCH_N(N, CALL)        \
    switch (N) {                          \
        case 16: return CALL(16);         \
        case 32: return CALL(32);         \
        case 64: return CALL(64);         \
        case 128: return CALL(128);       \
        case 256: return CALL(256);       \
        case 512: return CALL(512);       \
        case 1024: return CALL(1024);     \
        default: return cudaErrorInvalidValue; \
    }

// The real filtered fields of a window batch (the 3PCF monopole's shell fields): the window
// pass, the inverse y pass (radix-8 forms) and the c2r z pass of every window, stored.
template <int N>
static cudaError_t filtered_impl(const float2* spec, float2* work, float* out, const WinBatch& wb, const Tables& tb,
                                 cudaStream_t st, const Tracer& tr) {
    using C = Cfg<N>;
    cudaError_t e;
    if ((e = allow_smem(k_inv_z_c2r_store<N>, C::SMEM_Z)) != cudaSuccess) return e;
    tr(K_INV_X_WINDOW, 0, st);
    if ((e = launch_inv_x<N>(0, spec, work, wb, tb, 1, st)) != cudaSuccess) return e;
    tr(K_INV_X_WINDOW, 1, st);
    tr(K_INV_Y, 0, st);
    if ((e = launch_inv_y<N>(0, work, wb.S, tb.tw, st)) != cudaSuccess) return e;
    tr(K_INV_Y, 1, st);
    const float scale = 1.0f / ((float)N * (float)N * (float)N);
    for (int s = 0; s < wb.S; ++s) {
        tr(K_INV_Z_STORE, 0, st);
        k_inv_z_c2r_store<N><<<(N * N) / C::LZ, C::ZTHREADS, C::SMEM_Z, st>>>(
            work + (size_t)s * N * N * (N / 2), out + (size_t)s * N * N * N, scale, tb.tw);
        tr(K_INV_Z_STORE, 1, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_filtered_fields(int N, const float2* spec, float2* work, float* out, const WinBatch& wb,
                                   const Tables& tb, cudaStream_t st, const Tracer& tr) {
    if (wb.S < 1 || wb.S > 16 || (reinterpret_cast<uintptr_t>(wb.tab) & 15)) return cudaErrorInvalidValue;
#define F(n) filtered_impl<n>(spec, work, out, wb, tb, st, tr)
    HERMES_DISPATCH_N(N, F)
#undef F
}

cudaError_t launch_smooth_field(int N, const float2* spec, float2* work, float* out, const WinBatch& wb,
                                const Tables& tb, cudaStream_t st, const Tracer& tr) {
    if (wb.S != 1) return cudaErrorInvalidValue;
#define F(n) smooth_impl<n>(spec, work, out, wb, tb, st, tr)
    HERMES_DISPATCH_N(N, F)
#undef F
}

cudaError_t launch_forward(int N, float* grid, float2* spec, const double* scal, const Tables& tb, cudaStream_t st,
                           const Tracer& tr, int ncat) {
    if (ncat < 1 || ncat > MAX_CATALOGUES) return cudaErrorInvalidValue;
#define F(n) forward_impl<n>(grid, spec, scal, 1, tb, st, tr, ncat)
    HERMES_DISPATCH_N(N, F)
#undef F
}

cudaError_t launch_delta_to_spec(int N, float* grid, float2* spec, const double* scal, const Tables& tb,
                                 cudaStream_t st, const Tracer& tr, int keep_dc) {
#define F(n) forward_impl<n>(grid, spec, scal, 0, tb, st, tr, 1, keep_dc)
    HERMES_DISPATCH_N(N, F)
#undef F
}

cudaError_t launch_inverse_xi(int N, const float2* spec, float2* work, const float* delta, const WinBatch& wb,
                              const Tables& tb, double* dd_part, unsigned* err, cudaStream_t st, const Tracer& tr,
                              int ncat) {
    if (ncat < 1 || ncat > MAX_CATALOGUES || (size_t)wb.S * ncat > 65535) return cudaErrorInvalidValue;
#define F(n) inverse_impl<n>(spec, work, delta, wb, tb, dd_part, err, st, tr, ncat)
    HERMES_DISPATCH_N(N, F)
#undef F
}

static int x_blocks_of(int N) {
    switch (N) {
        case 16: return (8 / Cfg<16>::W) * 16;
        case 32: return (16 / Cfg<32>::W) * 32;
        case 64: return (32 / Cfg<64>::W) * 64;
        case 128: return (64 / Cfg<128>::W) * 128;
        case 256: return (128 / Cfg<256>::W) * 256;
        case 512: return (256 / Cfg<512>::W) * 512;
        case 1024: return (512 / Cfg<1024>::W) * 1024;
    }
    return 0;
}
static int z_blocks_of(int N) {
    switch (N) {
        case 16: return 256 / Cfg<16>::LZ;
        case 32: return 1024 / Cfg<32>::LZ;
        case 64: return 4096 / Cfg<64>::LZ;
        case 128: return 16384 / Cfg<128>::LZ;
        case 256: return 65536 / Cfg<256>::LZ;
        case 512: return 262144 / Cfg<512>::LZ;
        case 1024: return 1048576 / Cfg<1024>::LZ;
    }
    return 0;
}

int inv_z_blocks_plain(int N) { return z_blocks_of(N); }
int inv_x_blocks(int N) { return x_blocks_of(N); }
int inv_z_blocks(int N) {
    switch (N) {
        case 16: return yz_fused_ok<16>() ? 16 * YZCfg<16>::CL : z_blocks_of(N);
        case 32: return yz_fused_ok<32>() ? 32 * YZCfg<32>::CL : z_blocks_of(N);
        case 64: return yz_fused_ok<64>() ? 64 * YZCfg<64>::CL : z_blocks_of(N);
        case 128: return yz_fused_ok<128>() ? 128 * YZCfg<128>::CL : z_blocks_of(N);
        case 256: return yz_fused_ok<256>() ? 256 * YZCfg<256>::CL : z_blocks_of(N);
        case 512: return yz_fused_ok<512>() ? 512 * YZCfg<512>::CL : z_blocks_of(N);
    }
    return z_blocks_of(N);
}

}  // namespace hermes
