// fast_fft.cuh -- compile-time-sized FFT pieces for power-of-two grids.
//
// The zero-padded transforms of the demag convolution (Sec. 2, steps (1)-(5);
// Sec. 3, Eqs. (14)-(16)) have padded length L = 2n on an axis of n cells
// with only n nonzero inputs (forward) or n wanted outputs (inverse).  With
// W_L = exp(-2 pi i / L):
//   forward:  X[2m]   = FFT_n(x)[m],   X[2m+1] = FFT_n(x_j W_L^j)[m]
//   inverse:  x[j]    = IFFT_n(X_even)[j] + W_L^{-j} IFFT_n(X_odd)[j], j < n
// so every padded transform is two unpadded length-n FFTs: the zero half is
// never touched.
//
// An FFT of length n = P*Q runs on a group of max(P, Q) threads in two
// register steps and one shared-memory transpose:
//   step A: thread t < Q holds x[t + Q p], p < P; DFT_P over p; twiddle by
//           W_n^{t a}; store to ex[a][t]
//   step B: thread a < P holds ex[a][t], t < Q; DFT_Q over t gives
//           X[a + P b], b < Q.
// Inverse transforms conjugate in and out.  Twiddles come from a shared
// table tw[k] = W_L^k, k < L = 2n (so W_n^k = tw[2k]).
#pragma once
#include "fft_device.cuh"

namespace mmk {

__device__ __forceinline__ void dft32(float2* a) {
    float2 e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        e[i] = a[2 * i];
        o[i] = a[2 * i + 1];
    }
    dft16(e);
    dft16(o);
    // o_q *= W_32^q = cos(pi q/16) - i sin(pi q/16), q < 16 (mathematical constants)
    constexpr float c[16] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f, 0.83146961230254523708f,
                             0.70710678118654752440f, 0.55557023301960222474f, 0.38268343236508977173f,
                             0.19509032201612826785f, 0.0f, -0.19509032201612826785f, -0.38268343236508977173f,
                             -0.55557023301960222474f, -0.70710678118654752440f, -0.83146961230254523708f,
                             -0.92387953251128675613f, -0.98078528040323044913f};
    constexpr float s[16] = {0.0f, 0.19509032201612826785f, 0.38268343236508977173f, 0.55557023301960222474f,
                             0.70710678118654752440f, 0.83146961230254523708f, 0.92387953251128675613f,
                             0.98078528040323044913f, 1.0f, 0.98078528040323044913f, 0.92387953251128675613f,
                             0.83146961230254523708f, 0.70710678118654752440f, 0.55557023301960222474f,
                             0.38268343236508977173f, 0.19509032201612826785f};
#pragma unroll
    for (int q = 1; q < 16; ++q) o[q] = cmul(o[q], make_float2(c[q], -s[q]));
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        a[q] = cadd(e[q], o[q]);
        a[q + 16] = csub(e[q], o[q]);
    }
}

template <int R> __device__ __forceinline__ void dftp(float2* a);
template <> __device__ __forceinline__ void dftp<1>(float2*) {}
template <> __device__ __forceinline__ void dftp<2>(float2* a) { dft2(a); }
template <> __device__ __forceinline__ void dftp<4>(float2* a) { dft4(a); }
template <> __device__ __forceinline__ void dftp<8>(float2* a) { dft8(a); }
template <> __device__ __forceinline__ void dftp<16>(float2* a) { dft16(a); }
template <> __device__ __forceinline__ void dftp<32>(float2* a) { dft32(a); }

// Split of n into P x Q for the two register steps.
template <int N> struct Split;
template <> struct Split<8> { static constexpr int P = 4, Q = 2; };
template <> struct Split<16> { static constexpr int P = 4, Q = 4; };
template <> struct Split<32> { static constexpr int P = 8, Q = 4; };
template <> struct Split<64> { static constexpr int P = 8, Q = 8; };
template <> struct Split<128> { static constexpr int P = 16, Q = 8; };
template <> struct Split<256> { static constexpr int P = 16, Q = 16; };
template <> struct Split<512> { static constexpr int P = 16, Q = 32; };
template <> struct Split<1024> { static constexpr int P = 32, Q = 32; };

template <int N> struct Fft2 {
    static constexpr int P = Split<N>::P;
    static constexpr int Q = Split<N>::Q;
    static constexpr int G = P > Q ? P : Q;        // threads per transform
    static constexpr int EXS = Q + 1;              // padded exchange row
    static constexpr int EX = P * EXS;             // exchange buffer (complex)

    // Step A on v[p] = x[t + Q p] (t < Q): DFT_P, twiddle W_N^{t a}, store.
    // tw: W_{2N}^k table.  conj_in conjugates the input first.
    static __device__ __forceinline__ void stepA(float2 (&v)[P], int t, const float2* tw, float2* ex,
                                                 bool conj_in) {
        if (conj_in) {
#pragma unroll
            for (int p = 0; p < P; ++p) v[p].y = -v[p].y;
        }
        dftp<P>(v);
#pragma unroll
        for (int a = 1; a < P; ++a) v[a] = cmul(v[a], tw[2 * t * a]);
#pragma unroll
        for (int a = 0; a < P; ++a) ex[a * EXS + t] = v[a];
    }

    // Step B for thread a < P: gather ex[a][t], DFT_Q; w[b] = X[a + P b].
    static __device__ __forceinline__ void stepB(float2 (&w)[Q], int a, const float2* ex, bool conj_out) {
#pragma unroll
        for (int t = 0; t < Q; ++t) w[t] = ex[a * EXS + t];
        dftp<Q>(w);
        if (conj_out) {
#pragma unroll
            for (int b = 0; b < Q; ++b) w[b].y = -w[b].y;
        }
    }
};

}  // namespace mmk
