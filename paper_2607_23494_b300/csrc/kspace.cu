// k-space (Parseval) route for xi, xi_l and the axisymmetric xi(r_perp, r_par),
// Eq. (pair-counting-kspace):
//   (1/N^3) sum_x delta delta~_b = (1/N^6) sum_n |delta^_n|^2 K_b(n),
// and the self-pair term (1/(N^6 eps_bar^2)) sum_n K_b(n) S^(n).  Every window
// of this library has K_{b,l}(n) = c_l T_{b,l}(|n|^2) Phi^(n) L_l(k_z/k), so one
// pass over the half spectrum builds, for each requested l, the float64 radial
// histogram
//   A_l(q) = sum_{|n|^2 = q} w_z Phi^(n) L_l(mu_n) (|delta^_n|^2 - S^(n) / eps_bar^2)
// (w_z = 1 for k_z = 0, 2 for 0 < k_z < N/2; Nyquist modes carry K = 0), and
//   xi_{b,l} = c_l sum_q T_{b,l}(q) A_l(q) / N^6.
// delta^ is read once for every window of every order.
#include "kernels.h"
#include "fft_core.cuh"

namespace hermes {

template <int N>
struct KsCfg {
    static constexpr int H = N / 2;
    static constexpr int W = (N / 2 < 16) ? N / 2 : 16;  // k_z columns per block
    static constexpr int TX = 256 / W;                   // threads along k_x
    static constexpr int THREADS = TX * W;
};

__device__ __forceinline__ float legendre_k(int ell, float mu) {
    if (ell == 0) return 1.0f;
    float p0 = 1.0f, p1 = mu;
    for (int n = 1; n < ell; ++n) {
        const float p2 = ((float)(2 * n + 1) * mu * p1 - (float)n * p0) / (float)(n + 1);
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

// Exact float32 -> float64 widening done with integer instructions (IEEE 754
// binary32 -> binary64: re-bias the exponent by 1023 - 127 = 896 and left-align
// the 23-bit fraction in the 52-bit one).  Subnormal inputs flush to signed
// zero (|v| < 1.2e-38 is far below any histogram entry that matters); Inf/NaN
// keep their class.  This keeps the conversion off the float64 pipe.
__device__ __forceinline__ double widen_f32(float v) {
    const unsigned u = __float_as_uint(v);
    const unsigned sign = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    if (e == 0) return __hiloint2double((int)sign, 0);
    const unsigned e64 = (e == 0xffu) ? 0x7ffu : e + 896u;
    return __hiloint2double((int)(sign | (e64 << 20) | (m >> 3)), (int)(m << 29));
}

// Block (k_z chunk, k_y in [0, N/2)); thread (col, tx) walks k_x = tx, tx + TX, ... < N/2.
// The mirror modes (+-n_x, +-n_y) share |n|^2, Phi^ and S^ (both even in every
// component), so a thread sums |delta^|^2 over the up to four of them that are
// stored and issues one atomic per order instead of four.
// SELF: only the self-pair part, B_l(q) = sum_{|n|^2=q} w_z Phi^(n) L_l(mu) S^(n)
// (positive, not divided by eps_bar^2; the spectrum is not read).
template <int N, bool SELF>
__global__ void __launch_bounds__(KsCfg<N>::THREADS) k_kspace_hist(const float2* __restrict__ spec, const Tables tb,
                                                                   int P, const double* __restrict__ scal,
                                                                   KsOrders ko, double* __restrict__ hist,
                                                                   int64_t Q) {
    using C = KsCfg<N>;
    constexpr int W = C::W, TX = C::TX, H = N / 2;
    const int col = threadIdx.x % W, tx = threadIdx.x / W;
    const int ky = blockIdx.y, kz = blockIdx.x * W + col;
    const int ky2 = (N - ky) & (N - 1);  // mirror row (== ky for ky = 0)
    const int ny = ky, nz = kz;
    const float phyz = __ldg(tb.phi + ky) * __ldg(tb.phi + kz);
    const double inv_eps2 = SELF ? 0.0 : scal[2] * scal[2];  // scal[2] = N^3 / sum w = 1 / eps_bar
    // self-pair transform S^(n) = sum_a C(k_x, a) U[a], U[a] = sum_{b,c} S(a,b,c) C(k_y,b) C(k_z,c)
    float cy[8], cz[8], U[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        cy[a] = (a == 0) ? 1.0f : 2.0f * __ldg(tb.tw + N + ((ky * a) & (N - 1))).x;
        cz[a] = (a == 0) ? 1.0f : 2.0f * __ldg(tb.tw + N + ((kz * a) & (N - 1))).x;
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        float u = 0.0f;
        if (a < P) {
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                if (b < P) {
                    float ub = 0.0f;
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (c < P) ub = fmaf(__ldg(tb.stab + (a * P + b) * P + c), cz[c], ub);
                    u = fmaf(ub, cy[b], u);
                }
            }
        }
        U[a] = u;
    }
    // Per-mode arithmetic in float32 (B300's float64 issue rate is a small
    // fraction of float32's); only the histogram accumulates in float64.
    const float wz = (kz == 0) ? 1.0f : 2.0f;
    const float ny_cnt = (ky == 0) ? 1.0f : 2.0f;
    const float inv_e2 = (float)inv_eps2;
    for (int kx = tx; kx < H; kx += TX) {
        const int kx2 = (N - kx) & (N - 1);
        const int qp = kx * kx + ny * ny;  // mirrors share n_x^2 + n_y^2 and |n_z|
        const int q = qp + nz * nz;
        float pw = 0.0f;
        if constexpr (!SELF) {
            const float2 d00 = spec[((size_t)kx * N + ky) * H + kz];
            pw = fmaf(d00.x, d00.x, d00.y * d00.y);
            if (ky) {
                const float2 d = spec[((size_t)kx * N + ky2) * H + kz];
                pw += fmaf(d.x, d.x, d.y * d.y);
            }
            if (kx) {
                const float2 d = spec[((size_t)kx2 * N + ky) * H + kz];
                pw += fmaf(d.x, d.x, d.y * d.y);
                if (ky) {
                    const float2 e = spec[((size_t)kx2 * N + ky2) * H + kz];
                    pw += fmaf(e.x, e.x, e.y * e.y);
                }
            }
        }
        float sh = 0.0f;
#pragma unroll
        for (int a = 0; a < 8; ++a)
            if (a < P) sh = fmaf((a == 0) ? 1.0f : 2.0f * __ldg(tb.tw + N + ((kx * a) & (N - 1))).x, U[a], sh);
        const float cnt = ny_cnt * ((kx == 0) ? 1.0f : 2.0f);
        pw = SELF ? cnt * sh : fmaf(-cnt * sh, inv_e2, pw);
        const float base = wz * (__ldg(tb.phi + kx) * phyz) * pw;
        const float mu = q > 0 ? (float)nz * rsqrtf((float)q) : 0.0f;
        for (int o = 0; o < ko.n; ++o) {
            const float f = ko.cyl ? __ldg(ko.par + ko.ell[o] * H + nz)
                                   : (ko.ell[o] == 0 ? 1.0f : legendre_k(ko.ell[o], mu));
            const float v = base * f;
            atomicAdd(hist + (size_t)o * Q + (ko.cyl ? qp : q), widen_f32(v));
        }
    }
}

// out[o][b] += c_l sum_q T[(l*Q + q)*nbp + b] * hist[o*Q + q] / N^6 (out zeroed first).
// Grid (q slices, 32-bin chunks, orders); lane = bin within the chunk, so every
// warp reads table rows contiguously.  A warp takes 32 consecutive q at a time:
// each lane narrows one histogram entry to float32 and the warp shares them by
// shuffles; the 32 products accumulate in float32 and each group of 32 is added
// into a float64 sum, so float64 work is one add per 32 table entries.
constexpr int KC_THREADS = 256;
__global__ void __launch_bounds__(KC_THREADS) k_kspace_contract(const float* __restrict__ rad, int nbp, int64_t Q,
                                                                KsOrders ko, const double* __restrict__ hist,
                                                                double n6, double* __restrict__ out, int nb) {
    __shared__ double part[KC_THREADS / 32][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int o = blockIdx.z, b = blockIdx.y * 32 + lane;
    const int ell = ko.ell[o];
    const bool live = b < nb;
    // isotropic: the table block of order l; axisymmetric: the one transverse table
    const float* tab = rad + (ko.cyl ? 0 : (size_t)ell * Q * nbp) + (live ? b : 0);
    const double* h = hist + (size_t)o * Q;
    const int64_t ngroups = (Q + 31) / 32;
    const int64_t nwarps = (int64_t)gridDim.x * (KC_THREADS / 32);
    double s = 0.0;
    for (int64_t g = (int64_t)blockIdx.x * (KC_THREADS / 32) + wid; g < ngroups; g += nwarps) {
        const int64_t q0 = g * 32;
        const int64_t qn = (Q - q0) < 32 ? (Q - q0) : 32;
        const float hl = lane < qn ? (float)__ldg(h + q0 + lane) : 0.0f;
        float acc = 0.0f;
        if (qn == 32) {
#pragma unroll 8
            for (int j = 0; j < 32; ++j) {
                const float hj = __shfl_sync(0xffffffffu, hl, j);
                acc = fmaf(__ldg(tab + (size_t)(q0 + j) * nbp), hj, acc);
            }
        } else {
            for (int j = 0; j < qn; ++j) {
                const float hj = __shfl_sync(0xffffffffu, hl, j);
                acc = fmaf(__ldg(tab + (size_t)(q0 + j) * nbp), hj, acc);
            }
        }
        s += (double)acc;
    }
    part[wid][lane] = s;
    __syncthreads();
    if (wid == 0) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < KC_THREADS / 32; ++w) t += part[w][lane];
        if (live) {
            const double c = ko.cyl ? 1.0 : (double)(2 * ell + 1) * (((ell / 2) & 1) ? -1.0 : 1.0);
            atomicAdd(out + (size_t)o * nb + b, c * t / n6);
        }
    }
}

// Ring windows: out[o] = sum_q T[q*nbp + ell[o]] hist[o*Q + q] / N^6, one column per
// entry.  Grid (q slices, entries); lane j of a warp takes q0 + j, products in float32
// per group of 32 q, summed across the warp and added in float64.
__global__ void __launch_bounds__(KC_THREADS) k_kspace_contract_diag(const float* __restrict__ rad, int nbp,
                                                                     int64_t Q, KsOrders ko,
                                                                     const double* __restrict__ hist, double n6,
                                                                     double* __restrict__ out) {
    __shared__ double part[KC_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int o = blockIdx.y;
    const float* tab = rad + ko.ell[o];
    const double* h = hist + (size_t)o * Q;
    const int64_t ngroups = (Q + 31) / 32;
    const int64_t nwarps = (int64_t)gridDim.x * (KC_THREADS / 32);
    double s = 0.0;
    for (int64_t g = (int64_t)blockIdx.x * (KC_THREADS / 32) + wid; g < ngroups; g += nwarps) {
        const int64_t q = g * 32 + lane;
        float acc = q < Q ? __ldg(tab + (size_t)q * nbp) * (float)__ldg(h + q) : 0.0f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        s += (double)acc;
    }
    if (lane == 0) part[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < KC_THREADS / 32; ++w) t += part[w];
        atomicAdd(out + o, t / n6);
    }
}

template <int N>
static cudaError_t kspace_impl(const float2* spec, const Tables& tb, int P, const double* scal, const KsOrders& ko,
                               double* hist, int64_t Q, cudaStream_t st, const Tracer& tr, int self_only) {
    using C = KsCfg<N>;
    dim3 g((N / 2) / C::W, N / 2, 1);
    tr(self_only ? K_SN_HIST : K_KSPACE_HIST, 0, st);
    if (self_only) k_kspace_hist<N, true><<<g, C::THREADS, 0, st>>>(spec, tb, P, scal, ko, hist, Q);
    else k_kspace_hist<N, false><<<g, C::THREADS, 0, st>>>(spec, tb, P, scal, ko, hist, Q);
    tr(self_only ? K_SN_HIST : K_KSPACE_HIST, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_kspace_hist(int N, const float2* spec, const Tables& tb, int P, const double* scal,
                               const KsOrders& ko, double* hist, int64_t Q, cudaStream_t st, const Tracer& tr,
                               int self_only) {
    switch (N) {
        case 16: return kspace_impl<16>(spec, tb, P, scal, ko, hist, Q, st, tr, self_only);
        case 32: return kspace_impl<32>(spec, tb, P, scal, ko, hist, Q, st, tr, self_only);
        case 64: return kspace_impl<64>(spec, tb, P, scal, ko, hist, Q, st, tr, self_only);
        case 128: return kspace_impl<128>(spec, tb, P, scal, ko, hist, Q, st, tr, self_only);
        case 256: return kspace_impl<256>(spec, tb, P, scal, ko, hist, Q, st, tr, self_only);
        case 512: return kspace_impl<512>(spec, tb, P, scal, ko, hist, Q, st, tr, self_only);
        case 1024: return kspace_impl<1024>(spec, tb, P, scal, ko, hist, Q, st, tr, self_only);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_kspace_contract(const float* rad, int nbp, int64_t Q, const KsOrders& ko, const double* hist,
                                   int N, double* out, int nb, cudaStream_t st, const Tracer& tr, int trace_id) {
    const double n3 = (double)N * N * N;
    if (ko.diag) {
        const int64_t groups = (Q + 31) / 32;
        const int64_t most = (groups + KC_THREADS / 32 - 1) / (KC_THREADS / 32);
        const int64_t want = (4 * 148 + ko.n - 1) / ko.n;
        const int slices = (int)(want < most ? want : most);
        tr(trace_id, 0, st);
        cudaError_t e = cudaMemsetAsync(out, 0, (size_t)ko.n * sizeof(double), st);
        if (e != cudaSuccess) return e;
        k_kspace_contract_diag<<<dim3(slices, ko.n), KC_THREADS, 0, st>>>(rad, nbp, Q, ko, hist, n3 * n3, out);
        tr(trace_id, 1, st);
        return cudaGetLastError();
    }
    const int chunks = (nb + 31) / 32;
    // about four blocks per SM in total, but at least one group of 32 q per warp
    const int64_t groups = (Q + 31) / 32;
    const int64_t most = (groups + KC_THREADS / 32 - 1) / (KC_THREADS / 32);
    int64_t want = (4 * 148 + chunks * ko.n - 1) / (chunks * ko.n);
    const int slices = (int)(want < most ? want : most);
    tr(trace_id, 0, st);
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)ko.n * nb * sizeof(double), st);
    if (e != cudaSuccess) return e;
    k_kspace_contract<<<dim3(slices, chunks, ko.n), KC_THREADS, 0, st>>>(rad, nbp, Q, ko, hist, n3 * n3, out, nb);
    tr(trace_id, 1, st);
    return cudaGetLastError();
}

}  // namespace hermes
