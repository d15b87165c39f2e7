// Shared-memory Stockham FFT on one line of length M held by M/8 threads.
//
// Every thread owns 8 complex values.  Before and after the transform thread t
// holds elements t + i*T (i = 0..7, T = M/8) of its line, so the first stage
// can be fed straight from coalesced global loads and the last stage can be
// stored (or contracted) straight from registers.  Intermediate stages
// exchange data through shared memory; the layout of a line in shared memory
// is a policy class (strided tiles vs. contiguous padded lines).
//
// Stage plan: radix-8 throughout, with one leading radix-2 or radix-4 stage
// when log2(M) is not a multiple of 3.  Twiddles come from tables built on the
// host in float64 and laid out so each load is coalesced; the inverse uses
// conjugates.
#pragma once
#include "common.cuh"

namespace hermes {

template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {  // forward: -i a ; inverse: +i a
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2* a) {
    float2 t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
    float2 s13 = cadd(a1, a3), d13 = csub(a1, a3);
    float2 t = mul_mi<INV>(d13);
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = cadd(d02, t);
    a3 = csub(d02, t);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2* a) { dft4<INV>(a[0], a[1], a[2], a[3]); }

template <bool INV>
__device__ __forceinline__ void dft8(float2* a) {
    const float r = 0.70710678118654752440f;
    float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    float2 o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    // o_k *= w8^k, w8 = e^{-+ 2 pi i / 8}
    float2 w1, w2, w3;
    if (!INV) {
        w1 = make_float2((o1.x + o1.y) * r, (o1.y - o1.x) * r);
        w3 = make_float2((o3.y - o3.x) * r, -(o3.x + o3.y) * r);
    } else {
        w1 = make_float2((o1.x - o1.y) * r, (o1.x + o1.y) * r);
        w3 = make_float2(-(o3.x + o3.y) * r, (o3.x - o3.y) * r);
    }
    w2 = mul_mi<INV>(o2);
    a[0] = cadd(e0, o0);
    a[4] = csub(e0, o0);
    a[1] = cadd(e1, w1);
    a[5] = csub(e1, w1);
    a[2] = cadd(e2, w2);
    a[6] = csub(e2, w2);
    a[3] = cadd(e3, w3);
    a[7] = csub(e3, w3);
}

template <int R, bool INV>
__device__ __forceinline__ void dftR(float2* a) {
    if constexpr (R == 2) dft2<INV>(a);
    else if constexpr (R == 4) dft4<INV>(a);
    else dft8<INV>(a);
}

// Twiddle tables (one buffer, built on the host in float64, stored as float32):
//   tw[L + j]                       = e^{-2 pi i j / L},  L = 2, 4, ..., TW, 0 <= j < L
//   tw[STAGE_TW + 7 (NS-1) + (r-1) NS + k] = e^{-2 pi i k r / (8 NS)}, 1 <= r < 8, 0 <= k < NS
// The second block serves the radix-8 Stockham stages: for a fixed r the
// twiddles of consecutive butterflies are adjacent, so every load is coalesced
// and exact to float32 rounding.
constexpr int STAGE_TW = 2 * TW;
constexpr int TW_ENTRIES = STAGE_TW + 7 * TW;
template <bool INV>
__device__ __forceinline__ float2 twiddle_l(const float2* __restrict__ tw, int L, int j) {
    float2 w = __ldg(tw + L + j);
    return INV ? make_float2(w.x, -w.y) : w;
}
template <bool INV>
__device__ __forceinline__ float2 twiddle_stage8(const float2* __restrict__ tw, int NS, int r, int k) {
    float2 w = __ldg(tw + STAGE_TW + 7 * (NS - 1) + (r - 1) * NS + k);
    return INV ? make_float2(w.x, -w.y) : w;
}

// Shared-memory line layouts -------------------------------------------------
// Strided tile: W lines stored position-major, element (pos, col) at
// pos*W + col, plus 8 padding slots after every 8 rows.  With W = 8 the first
// exchange of a 512-point transform stores rows 8t + r from the four t of a warp;
// the 8-slot skew puts the two t of each half-warp on disjoint bank pairs (a
// 4-slot skew overlapped half of them: twice the minimum wavefronts).
template <int W>
struct SmemStrided {
    float2* p;
    int col;
    static constexpr int words(int n) { return n * W + (n / 8) * 8; }
    __device__ __forceinline__ int at(int pos) const { return pos * W + col + (pos >> 3) * 8; }
    __device__ __forceinline__ float2 ld(int pos) const { return p[at(pos)]; }
    __device__ __forceinline__ void st(int pos, float2 v) const { p[at(pos)] = v; }
    __device__ __forceinline__ static void sync() { __syncthreads(); }  // a tile spans the block
};
// Strided tile with a skew of P slots after every 2^SH rows, for the transforms
// at 16 or 32 values per thread, whose exchanges write runs of 2^k rows per warp
// (the skew that reaches the minimum wavefront count depends on M, E and W).
template <int W, int SH, int P>
struct SmemStridedSk {
    float2* p;
    int col;
    static constexpr int words(int n) { return n * W + (n >> SH) * P; }
    __device__ __forceinline__ int at(int pos) const { return pos * W + col + (pos >> SH) * P; }
    __device__ __forceinline__ float2 ld(int pos) const { return p[at(pos)]; }
    __device__ __forceinline__ void st(int pos, float2 v) const { p[at(pos)] = v; }
    __device__ __forceinline__ static void sync() { __syncthreads(); }
};
// Contiguous line of length M with one padding slot every 2^SH elements.
constexpr int line_shift(int m) { return m >= 128 ? 4 : (m == 32 ? 2 : 3); }
template <int M>
struct SmemLine {
    static constexpr int SH = line_shift(M);
    float2* p;
    __device__ __forceinline__ static int at(int pos) { return pos + (pos >> SH); }
    __device__ __forceinline__ float2 ld(int pos) const { return p[at(pos)]; }
    __device__ __forceinline__ void st(int pos, float2 v) const { p[at(pos)] = v; }
    __device__ __forceinline__ static void sync() { __syncthreads(); }
};
// A contiguous line whose M/8 threads are consecutive (thread group g =
// threadIdx.x / (M/8) of the block): its exchanges only wait for that group,
// so the other lines of the block run on.  Up to 32 threads that is their
// warp; above, named barrier 1 + g over the group's warps (at most 15 groups
// per block; barrier 0 stays the block-wide one).
template <int M>
struct SmemZLine : SmemLine<M> {
    int group;
    __device__ __forceinline__ void sync() const {
        if constexpr (M / 8 <= 32) __syncwarp();
        else asm volatile("bar.sync %0, %1;\n" ::"r"(1 + group), "n"(M / 8) : "memory");
    }
};
// The padded line of SmemLine for a line whose threads all belong to one warp (any
// length; the caller guarantees it): its exchanges only synchronise the warp.
template <int M>
struct SmemWarpLine : SmemLine<M> {
    __device__ __forceinline__ static void sync() { __syncwarp(); }
};
template <int M>
struct LinePad {
    static constexpr int value = M + (M >> line_shift(M)) + 1;
};

constexpr int ilog2c(int m) { return m <= 1 ? 0 : 1 + ilog2c(m >> 1); }
template <int M>
struct FirstRadix {
    static constexpr int lg = ilog2c(M);
    static constexpr int value = (lg % 3 == 0) ? 8 : (lg % 3 == 1 ? 2 : 4);
};

// x[r] *= w^r for r = 1..7 from w^1, w^2, w^4 (w^3, w^5, w^6, w^7 as products of at
// most two of them; relative error a few float32 ulps).
__device__ __forceinline__ void twiddle_from3(float2 (&x)[8], float2 w1, float2 w2, float2 w4) {
    const float2 w3 = cmul(w1, w2);
    x[1] = cmul(x[1], w1);
    x[2] = cmul(x[2], w2);
    x[3] = cmul(x[3], w3);
    x[4] = cmul(x[4], w4);
    x[5] = cmul(x[5], cmul(w1, w4));
    x[6] = cmul(x[6], cmul(w2, w4));
    x[7] = cmul(x[7], cmul(w3, w4));
}

// One Stockham stage.  v[u + r*U] is input r of butterfly b = t + u*T.
// TW7: load all seven radix-8 twiddles instead of three (for passes whose
// loads are already hidden and that are short of issue slots).
// WC: the twiddles w^1, w^2, w^4 of the thread's butterfly in every twiddled stage
// come preloaded in wc[3 (SI - 1) + {0, 1, 2}] (SI = index of the stage); with 8
// values per thread and radix 8 a thread's butterfly index is t in every such
// stage, so they are the same for every transform the thread runs.
template <int M, int R, int NS, bool INV, bool TW7, bool WC, int SI, class S>
__device__ __forceinline__ void fft_stage(float2 (&v)[8], int t, const float2* __restrict__ tw, const S& sm,
                                          const float2* wc) {
    constexpr int T = M / 8;
    constexpr int U = 8 / R;
    constexpr bool LAST = (NS * R == M);
    float2 out[8];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int b = t + u * T;
        const int k = b & (NS - 1);
        float2 x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = v[u + r * U];
        if constexpr (NS > 1 && WC) {
            static_assert(R == 8 && U == 1, "preloaded twiddles serve radix-8 stages of one butterfly per thread");
            twiddle_from3(x, wc[3 * (SI - 1)], wc[3 * (SI - 1) + 1], wc[3 * (SI - 1) + 2]);
        } else if constexpr (NS > 1 && TW7) {
            static_assert(R == 8, "only the leading stage may use radix 2 or 4");
#pragma unroll
            for (int r = 1; r < 8; ++r) x[r] = cmul(x[r], twiddle_stage8<INV>(tw, NS, r, k));
        } else if constexpr (NS > 1) {
            static_assert(R == 8, "only the leading stage may use radix 2 or 4");
            // three table loads instead of seven
            twiddle_from3(x, twiddle_stage8<INV>(tw, NS, 1, k), twiddle_stage8<INV>(tw, NS, 2, k),
                          twiddle_stage8<INV>(tw, NS, 4, k));
        }
        dftR<R, INV>(x);
#pragma unroll
        for (int r = 0; r < R; ++r) out[u + r * U] = x[r];
    }
    if constexpr (LAST) {
        // position b + r*NS = t + (u + r*U)*T: already in the canonical order
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = out[i];
    } else {
        sm.sync();  // everyone finished reading the previous contents
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int b = t + u * T;
            const int base = (b / NS) * NS * R + (b & (NS - 1));
#pragma unroll
            for (int r = 0; r < R; ++r) sm.st(base + r * NS, out[u + r * U]);
        }
        sm.sync();
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = sm.ld(t + i * T);
    }
}

template <int M, int NS, bool INV, bool TW7, bool WC, int SI, class S>
__device__ __forceinline__ void fft_stages(float2 (&v)[8], int t, const float2* __restrict__ tw, const S& sm,
                                           const float2* wc) {
    constexpr int R = (NS == 1) ? FirstRadix<M>::value : 8;
    fft_stage<M, R, NS, INV, TW7, WC, SI, S>(v, t, tw, sm, wc);
    if constexpr (NS * R < M) fft_stages<M, NS * R, INV, TW7, WC, SI + 1, S>(v, t, tw, sm, wc);
}

// Number of twiddled (NS > 1) stages of an M-point transform.
template <int M>
constexpr int twiddled_stages() {
    int n = 0;
    for (int ns = FirstRadix<M>::value; ns < M; ns *= 8) ++n;
    return n;
}
// Loads the w^1, w^2, w^4 of thread t's butterfly for every twiddled stage of an
// M-point transform (8 values per thread) into wc[3 * twiddled_stages<M>()].
template <int M, bool INV>
__device__ __forceinline__ void load_stage_twiddles(int t, const float2* __restrict__ tw, float2* wc) {
    int ns = FirstRadix<M>::value;
#pragma unroll
    for (int si = 0; si < twiddled_stages<M>(); ++si, ns *= 8) {
        const int k = t & (ns - 1);
        wc[3 * si] = twiddle_stage8<INV>(tw, ns, 1, k);
        wc[3 * si + 1] = twiddle_stage8<INV>(tw, ns, 2, k);
        wc[3 * si + 2] = twiddle_stage8<INV>(tw, ns, 4, k);
    }
}

// In-register/shared FFT of length M (8 <= M <= TW).  Precondition: v[i] =
// x[t + i*M/8].  Postcondition: v[i] = X[t + i*M/8], X_k = sum_n x_n
// e^{-+2 pi i k n / M} (unnormalised).  All threads that share the layout's
// synchronisation (the block, or the thread group of a SmemZLine) must call it the
// same number of times (it synchronises them when M > 8).
template <int M, bool INV, bool TW7 = false, class S>
__device__ __forceinline__ void fft_line(float2 (&v)[8], int t, const float2* __restrict__ tw, const S& sm) {
    static_assert(M >= 8 && (M & (M - 1)) == 0 && M <= TW, "unsupported FFT length");
    fft_stages<M, 1, INV, TW7, false, 0, S>(v, t, tw, sm, nullptr);
}

// The same with the stage twiddles preloaded by load_stage_twiddles<M, INV>.
template <int M, bool INV, class S>
__device__ __forceinline__ void fft_line_wc(float2 (&v)[8], int t, const float2* __restrict__ tw, const S& sm,
                                            const float2* wc) {
    static_assert(M >= 8 && (M & (M - 1)) == 0 && M <= TW, "unsupported FFT length");
    fft_stages<M, 1, INV, false, true, 0, S>(v, t, tw, sm, wc);
}


// K lines per thread at once (8 values each), all exchanging behind the same
// barriers: one barrier pair per stage serves the K transforms, and the K
// butterflies between barriers are independent.  sms[k] is line k's layout; the
// stage twiddles come preloaded (load_stage_twiddles), so every twiddled stage
// must run one butterfly per thread.
template <int M, int R, int NS, bool INV, int SI, class S, int K>
__device__ __forceinline__ void fft_stage_k(float2 (&v)[K][8], int t, const S* sms, const float2* wc) {
    constexpr int T = M / 8;
    constexpr int U = 8 / R;
    constexpr bool LAST = (NS * R == M);
    float2 out[K][8];
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float2 x[R];
#pragma unroll
            for (int r = 0; r < R; ++r) x[r] = v[k][u + r * U];
            if constexpr (NS > 1) {
                static_assert(R == 8 && U == 1, "preloaded twiddles serve radix-8 stages of one butterfly per thread");
                twiddle_from3(x, wc[3 * (SI - 1)], wc[3 * (SI - 1) + 1], wc[3 * (SI - 1) + 2]);
            }
            dftR<R, INV>(x);
#pragma unroll
            for (int r = 0; r < R; ++r) out[k][u + r * U] = x[r];
        }
    }
    if constexpr (LAST) {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int i = 0; i < 8; ++i) v[k][i] = out[k][i];
    } else {
        sms[0].sync();
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int b = t + u * T;
                const int base = (b / NS) * NS * R + (b & (NS - 1));
#pragma unroll
                for (int r = 0; r < R; ++r) sms[k].st(base + r * NS, out[k][u + r * U]);
            }
        sms[0].sync();
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int i = 0; i < 8; ++i) v[k][i] = sms[k].ld(t + i * T);
    }
}
template <int M, int NS, bool INV, int SI, class S, int K>
__device__ __forceinline__ void fft_stages_k(float2 (&v)[K][8], int t, const S* sms, const float2* wc) {
    constexpr int R = (NS == 1) ? FirstRadix<M>::value : 8;
    fft_stage_k<M, R, NS, INV, SI, S, K>(v, t, sms, wc);
    if constexpr (NS * R < M) fft_stages_k<M, NS * R, INV, SI + 1, S, K>(v, t, sms, wc);
}
template <int M, bool INV, int K, class S>
__device__ __forceinline__ void fft_lines_wc(float2 (&v)[K][8], int t, const S* sms, const float2* wc) {
    static_assert(M >= 8 && (M & (M - 1)) == 0 && M <= TW, "unsupported FFT length");
    fft_stages_k<M, 1, INV, 0, S, K>(v, t, sms, wc);
}

// ---------------------------------------------------------------------------
// The same Stockham scheme with E = 8, 16 or 32 values per thread (M/E threads
// per line): radix-E stages, after a leading radix-2^r stage when log2(M) is not a
// multiple of log2(E).  More values per thread means fewer shared-memory exchanges
// (a 256-point line: one at E = 16, two at E = 8; 1024 points: one at E = 32)
// for more registers per thread.  Before and after the transform thread t holds
// elements t + i*M/E, as in fft_line.

template <bool INV>
__device__ __forceinline__ float2 rot(float2 a, float c, float s) {  // a * e^{-+ i theta}, c = cos, s = sin
    return INV ? make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.y, c, a.x * s))
               : make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s));
}

// 16-point DFT: two 8-point DFTs of the even and odd samples joined with
// e^{-+2 pi i k / 16}, k = 0..7.
template <bool INV>
__device__ __forceinline__ void dft16(float2* a) {
    float2 e[8], o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        e[j] = a[2 * j];
        o[j] = a[2 * j + 1];
    }
    dft8<INV>(e);
    dft8<INV>(o);
    constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;  // cos, sin (pi / 8)
    constexpr float r2 = 0.70710678118654752440f;
    o[1] = rot<INV>(o[1], c1, s1);
    o[2] = rot<INV>(o[2], r2, r2);
    o[3] = rot<INV>(o[3], s1, c1);
    o[4] = mul_mi<INV>(o[4]);
    o[5] = rot<INV>(o[5], -s1, c1);
    o[6] = rot<INV>(o[6], -r2, r2);
    o[7] = rot<INV>(o[7], -c1, s1);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        a[k] = cadd(e[k], o[k]);
        a[k + 8] = csub(e[k], o[k]);
    }
}

// 32-point DFT: two 16-point DFTs joined with e^{-+2 pi i k / 32}, k = 0..15.
template <bool INV>
__device__ __forceinline__ void dft32(float2* a) {
    float2 e[16], o[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        e[j] = a[2 * j];
        o[j] = a[2 * j + 1];
    }
    dft16<INV>(e);
    dft16<INV>(o);
    // cos and sin of k pi / 16, k = 0..8
    constexpr float C[9] = {1.0f,
                            0.98078528040323044913f,
                            0.92387953251128675613f,
                            0.83146961230254523708f,
                            0.70710678118654752440f,
                            0.55557023301960222474f,
                            0.38268343236508977173f,
                            0.19509032201612826785f,
                            0.0f};
#pragma unroll
    for (int k = 1; k < 16; ++k) {
        if (k == 8) {
            o[8] = mul_mi<INV>(o[8]);
        } else if (k < 8) {
            o[k] = rot<INV>(o[k], C[k], C[8 - k]);
        } else {  // theta = k pi / 16 > pi / 2: cos = -sin((k - 8) pi / 16), sin = cos((k - 8) pi / 16)
            o[k] = rot<INV>(o[k], -C[16 - k], C[k - 8]);
        }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        a[k] = cadd(e[k], o[k]);
        a[k + 16] = csub(e[k], o[k]);
    }
}

template <int R, bool INV>
__device__ __forceinline__ void dftRE(float2* a) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) dft2<INV>(a);
    else if constexpr (R == 4) dft4<INV>(a);
    else if constexpr (R == 8) dft8<INV>(a);
    else if constexpr (R == 16) dft16<INV>(a);
    else dft32<INV>(a);
}

// Leading radix of an M-point transform at E values per thread (1: none).
template <int M, int E>
struct LeadRadix {
    static constexpr int value = 1 << (ilog2c(M) % ilog2c(E));
};

// Stage twiddles of a radix-R stage of span NS: e^{-+2 pi i k r / (R NS)}, read from
// the multi-level table (exact entries tw[L + k r], L = R NS).
template <int R, int NS, bool INV>
__device__ __forceinline__ void stage_twiddles(const float2* __restrict__ tw, int k, float2* w) {
#pragma unroll
    for (int r = 1; r < R; ++r) w[r - 1] = twiddle_l<INV>(tw, R * NS, k * r);
}

// Number of twiddled stages (NS > 1) and the twiddles a thread needs for all of them
// when it runs one butterfly per stage (U = 1 in every twiddled stage).
template <int M, int E>
constexpr int twiddled_stages_e() {
    int n = 0;
    for (int ns = LeadRadix<M, E>::value == 1 ? E : LeadRadix<M, E>::value; ns < M; ns *= E) ++n;
    return n;
}
template <int M, int E>
constexpr int stage_twiddle_count() {
    return twiddled_stages_e<M, E>() * (E - 1);
}

// PRE: the twiddles of the thread's butterfly come preloaded in wc (as written by
// load_stage_twiddles_e); otherwise they are read from the table in every stage.
template <int M, int E, int R, int NS, bool INV, bool PRE, int SI, class S>
__device__ __forceinline__ void fft_stage_e(float2 (&v)[E], int t, const float2* __restrict__ tw, const S& sm,
                                            const float2* wc) {
    constexpr int T = M / E;
    constexpr int U = E / R;
    constexpr bool LAST = (NS * R == M);
    float2 out[E];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int b = t + u * T;
        const int k = b & (NS - 1);
        float2 x[R];
#pragma unroll
        for (int r = 0; r < R; ++r) x[r] = v[u + r * U];
        if constexpr (NS > 1) {
            if constexpr (PRE) {
                static_assert(U == 1, "preloaded twiddles serve stages of one butterfly per thread");
#pragma unroll
                for (int r = 1; r < R; ++r) x[r] = cmul(x[r], wc[(E - 1) * (SI - 1) + r - 1]);
            } else {
                float2 w[R - 1];
                stage_twiddles<R, NS, INV>(tw, k, w);
#pragma unroll
                for (int r = 1; r < R; ++r) x[r] = cmul(x[r], w[r - 1]);
            }
        }
        dftRE<R, INV>(x);
#pragma unroll
        for (int r = 0; r < R; ++r) out[u + r * U] = x[r];
    }
    if constexpr (LAST) {
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = out[i];
    } else {
        sm.sync();
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int b = t + u * T;
            const int base = (b / NS) * NS * R + (b & (NS - 1));
#pragma unroll
            for (int r = 0; r < R; ++r) sm.st(base + r * NS, out[u + r * U]);
        }
        sm.sync();
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = sm.ld(t + i * T);
    }
}

template <int M, int E, int NS, bool INV, bool PRE, int SI, class S>
__device__ __forceinline__ void fft_stages_e(float2 (&v)[E], int t, const float2* __restrict__ tw, const S& sm,
                                             const float2* wc) {
    constexpr int L0 = LeadRadix<M, E>::value;
    constexpr int R = (NS == 1 && L0 > 1) ? L0 : E;
    fft_stage_e<M, E, R, NS, INV, PRE, SI, S>(v, t, tw, sm, wc);
    if constexpr (NS * R < M) fft_stages_e<M, E, NS * R, INV, PRE, SI + 1, S>(v, t, tw, sm, wc);
}

// Loads the twiddles of thread t's butterfly for every twiddled stage of an M-point
// transform at E values per thread into wc[stage_twiddle_count<M, E>()].
template <int M, int E, bool INV>
__device__ __forceinline__ void load_stage_twiddles_e(int t, const float2* __restrict__ tw, float2* wc) {
    int ns = LeadRadix<M, E>::value == 1 ? E : LeadRadix<M, E>::value;
#pragma unroll
    for (int si = 0; si < twiddled_stages_e<M, E>(); ++si, ns *= E) {
        const int k = t & (ns - 1);
#pragma unroll
        for (int r = 1; r < E; ++r) wc[(E - 1) * si + r - 1] = twiddle_l<INV>(tw, E * ns, k * r);
    }
}

// In-register/shared FFT of length M at E values per thread.  Precondition: v[i] =
// x[t + i*M/E].  Postcondition: v[i] = X[t + i*M/E] (unnormalised, sign as fft_line).
template <int M, int E, bool INV, class S>
__device__ __forceinline__ void fft_line_e(float2 (&v)[E], int t, const float2* __restrict__ tw, const S& sm) {
    static_assert(E == 8 || E == 16 || E == 32, "8, 16 or 32 values per thread");
    static_assert(M >= E && (M & (M - 1)) == 0 && M <= TW, "unsupported FFT length");
    fft_stages_e<M, E, 1, INV, false, 0, S>(v, t, tw, sm, nullptr);
}
template <int M, int E, bool INV, class S>
__device__ __forceinline__ void fft_line_e_wc(float2 (&v)[E], int t, const float2* __restrict__ tw, const S& sm,
                                              const float2* wc) {
    static_assert(E == 8 || E == 16 || E == 32, "8, 16 or 32 values per thread");
    static_assert(M >= E && (M & (M - 1)) == 0 && M <= TW, "unsupported FFT length");
    fft_stages_e<M, E, 1, INV, true, 0, S>(v, t, tw, sm, wc);
}

}  // namespace hermes
