// k-space (Parseval) route for xi and xi_l, Eq. (pair-counting-kspace):
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

// Block (k_z chunk, k_y); thread (col, tx) walks k_x = tx, tx + TX, ...
template <int N>
__global__ void __launch_bounds__(KsCfg<N>::THREADS) k_kspace_hist(const float2* __restrict__ spec, const Tables tb,
                                                                   int P, const double* __restrict__ scal,
                                                                   KsOrders ko, double* __restrict__ hist,
                                                                   int64_t Q) {
    using C = KsCfg<N>;
    constexpr int W = C::W, TX = C::TX, H = N / 2;
    const int col = threadIdx.x % W, tx = threadIdx.x / W;
    const int ky = blockIdx.y, kz = blockIdx.x * W + col;
    if (ky == H) return;  // Nyquist plane: K = 0 for every window
    const int ny = signed_freq(ky, N), nz = kz;
    const float phyz = __ldg(tb.phi + ky) * __ldg(tb.phi + kz);
    const double inv_eps2 = scal[2] * scal[2];  // scal[2] = N^3 / sum w = 1 / eps_bar
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
    const double wz = (kz == 0) ? 1.0 : 2.0;
    for (int kx = tx; kx < N; kx += TX) {
        if (kx == H) continue;
        const int nx = signed_freq(kx, N);
        const int q = nx * nx + ny * ny + nz * nz;
        const float2 d = spec[((size_t)kx * N + ky) * H + kz];
        float sh = 0.0f;
#pragma unroll
        for (int a = 0; a < 8; ++a)
            if (a < P) sh = fmaf((a == 0) ? 1.0f : 2.0f * __ldg(tb.tw + N + ((kx * a) & (N - 1))).x, U[a], sh);
        const double pw = (double)d.x * d.x + (double)d.y * d.y - (double)sh * inv_eps2;
        const double base = wz * (double)(__ldg(tb.phi + kx) * phyz) * pw;
        const float mu = q > 0 ? (float)nz * rsqrtf((float)q) : 0.0f;
        for (int o = 0; o < ko.n; ++o) {
            const double v = ko.ell[o] == 0 ? base : base * (double)legendre_k(ko.ell[o], mu);
            atomicAdd(hist + (size_t)o * Q + q, v);
        }
    }
}

// xi[o][b] = c_l sum_q T[(l*Q + q)*nbp + b] * hist[o*Q + q] / N^6; one block per (o, b).
__global__ void __launch_bounds__(256) k_kspace_contract(const float* __restrict__ rad, int nbp, int64_t Q,
                                                         KsOrders ko, const double* __restrict__ hist, double n6,
                                                         double* __restrict__ out, int nb) {
    __shared__ double red[8];
    const int o = blockIdx.x / nb, b = blockIdx.x % nb;
    const int ell = ko.ell[o];
    const float* tab = rad + (size_t)ell * Q * nbp + b;
    const double* h = hist + (size_t)o * Q;
    double s = 0.0;
    for (int64_t q = threadIdx.x; q < Q; q += blockDim.x) s += (double)tab[(size_t)q * nbp] * h[q];
    s = block_sum_double(s, red);
    if (threadIdx.x == 0) {
        const double c = (double)(2 * ell + 1) * (((ell / 2) & 1) ? -1.0 : 1.0);
        out[blockIdx.x] = c * s / n6;
    }
}

template <int N>
static cudaError_t kspace_impl(const float2* spec, const Tables& tb, int P, const double* scal, const KsOrders& ko,
                               double* hist, int64_t Q, cudaStream_t st, const Tracer& tr) {
    using C = KsCfg<N>;
    dim3 g((N / 2) / C::W, N, 1);
    tr(K_KSPACE_HIST, 0, st);
    k_kspace_hist<N><<<g, C::THREADS, 0, st>>>(spec, tb, P, scal, ko, hist, Q);
    tr(K_KSPACE_HIST, 1, st);
    return cudaGetLastError();
}

cudaError_t launch_kspace_hist(int N, const float2* spec, const Tables& tb, int P, const double* scal,
                               const KsOrders& ko, double* hist, int64_t Q, cudaStream_t st, const Tracer& tr) {
    switch (N) {
        case 16: return kspace_impl<16>(spec, tb, P, scal, ko, hist, Q, st, tr);
        case 32: return kspace_impl<32>(spec, tb, P, scal, ko, hist, Q, st, tr);
        case 64: return kspace_impl<64>(spec, tb, P, scal, ko, hist, Q, st, tr);
        case 128: return kspace_impl<128>(spec, tb, P, scal, ko, hist, Q, st, tr);
        case 256: return kspace_impl<256>(spec, tb, P, scal, ko, hist, Q, st, tr);
        case 512: return kspace_impl<512>(spec, tb, P, scal, ko, hist, Q, st, tr);
        case 1024: return kspace_impl<1024>(spec, tb, P, scal, ko, hist, Q, st, tr);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_kspace_contract(const float* rad, int nbp, int64_t Q, const KsOrders& ko, const double* hist,
                                   int N, double* out, int nb, cudaStream_t st, const Tracer& tr) {
    const double n3 = (double)N * N * N;
    tr(K_KSPACE_CONTRACT, 0, st);
    k_kspace_contract<<<ko.n * nb, 256, 0, st>>>(rad, nbp, Q, ko, hist, n3 * n3, out, nb);
    tr(K_KSPACE_CONTRACT, 1, st);
    return cudaGetLastError();
}

}  // namespace hermes
