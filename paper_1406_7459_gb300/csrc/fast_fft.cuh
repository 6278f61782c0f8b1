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
#include <cuda_pipeline.h>
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

// cos(pi k / 32) for k = 0..16 (mathematical constants); cospi32 / sinpi32
// extend it to any integer k by symmetry.  Used with compile-time k only.
__device__ __forceinline__ float cospi32(int k) {
    constexpr float q[17] = {1.0f, 0.99518472667219688624f, 0.98078528040323044913f, 0.95694033573220886494f,
                             0.92387953251128675613f, 0.88192126434835502971f, 0.83146961230254523708f,
                             0.77301045336273696081f, 0.70710678118654752440f, 0.63439328416364549822f,
                             0.55557023301960222474f, 0.47139673682599764856f, 0.38268343236508977173f,
                             0.29028467725446236764f, 0.19509032201612826785f, 0.09801714032956060199f, 0.0f};
    k &= 63;
    if (k <= 16) return q[k];
    if (k <= 32) return -q[32 - k];
    if (k <= 48) return -q[k - 32];
    return q[64 - k];
}
__device__ __forceinline__ float sinpi32(int k) { return cospi32(k - 16); }

// W_{2R}^q = exp(-i pi q / R) for compile-time q (R divides 32).
template <int R> __device__ __forceinline__ float2 wpi(int q) {
    return make_float2(cospi32(q * (32 / R)), -sinpi32(q * (32 / R)));
}

template <int N> struct Fft2 {
    static constexpr int P = Split<N>::P;
    static constexpr int Q = Split<N>::Q;
    static constexpr int G = P > Q ? P : Q;        // threads per transform
    static constexpr int EXS = Q + 1;              // padded exchange row
    static constexpr int EX = P * EXS;             // exchange buffer (complex)

    // w[a] = W_N^{t a}, a < P, from two table entries (W_N^t, W_N^{4t}) and
    // short product chains (at most ~P/4 + 2 rounded products per entry).
    // tw: W_{2N}^k table.
    static __device__ __forceinline__ void twiddles(int t, const float2* tw, float2 (&w)[P]) {
        w[0] = make_float2(1.f, 0.f);
        if (P > 1) w[1] = tw[2 * t];
        if (P > 2) w[2] = cmul(w[1], w[1]);
        if (P > 3) w[3] = cmul(w[2], w[1]);
        if (P > 4) {
            float2 w4m = tw[8 * t];                 // W_N^{4t}
#pragma unroll
            for (int m = 1; m < P / 4; ++m) {
                if (m > 1) w4m = cmul(w4m, tw[8 * t]);
                w[4 * m] = w4m;
                w[4 * m + 1] = cmul(w4m, w[1]);
                w[4 * m + 2] = cmul(w4m, w[2]);
                w[4 * m + 3] = cmul(w4m, w[3]);
            }
        }
    }

    // Step A on v[p] = x[t + Q p] (t < Q): DFT_P, twiddle by W_N^{t a};
    // the result stays in v.  conj_in conjugates the input first.
    static __device__ __forceinline__ void stepA_reg(float2 (&v)[P], int t, const float2* tw, bool conj_in) {
        if (conj_in) {
#pragma unroll
            for (int p = 0; p < P; ++p) v[p].y = -v[p].y;
        }
        dftp<P>(v);
        float2 w[P];
        twiddles(t, tw, w);
#pragma unroll
        for (int a = 1; a < P; ++a) v[a] = cmul(v[a], w[a]);
    }

    static __device__ __forceinline__ void store_ex(const float2 (&v)[P], int t, float2* ex) {
#pragma unroll
        for (int a = 0; a < P; ++a) ex[a * EXS + t] = v[a];
    }

    static __device__ __forceinline__ void stepA(float2 (&v)[P], int t, const float2* tw, float2* ex,
                                                 bool conj_in) {
        stepA_reg(v, t, tw, conj_in);
        store_ex(v, t, ex);
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

    // Table-driven variants for kernels that keep, besides tw, the table
    // ta[a Q + t] = W_N^{t a} (a < P, t < Q) in shared memory: every twiddle
    // is one conflict-free load (consecutive t read consecutive words).
    static __device__ __forceinline__ void stepA_tab(float2 (&v)[P], int t, const float2* ta, float2* ex,
                                                     bool conj_in) {
        if (conj_in) {
#pragma unroll
            for (int p = 0; p < P; ++p) v[p].y = -v[p].y;
        }
        dftp<P>(v);
#pragma unroll
        for (int a = 1; a < P; ++a) v[a] = cmul(v[a], ta[a * Q + t]);
        store_ex(v, t, ex);
    }
    // x_j *= W_{2N}^j, j = t + Q q
    static __device__ __forceinline__ void odd_input_tab(float2 (&v)[P], int t, const float2* tw) {
#pragma unroll
        for (int q = 0; q < P; ++q) v[q] = cmul(v[q], tw[t + Q * q]);
    }
    // y_n *= W_{2N}^{-n}, n = a + P b
    static __device__ __forceinline__ void odd_output_tab(float2 (&w)[Q], int a, const float2* tw) {
#pragma unroll
        for (int b = 0; b < Q; ++b) w[b] = cmul(w[b], cconj(tw[a + P * b]));
    }
    // Fill ta from the W_{2N} table in global memory (asynchronous 8-byte
    // copies; the caller commits and waits with its other prologue copies).
    // T: the block size.
    template <int T>
    static __device__ __forceinline__ void load_ta(float2* ta, const float2* tw_global) {
#pragma unroll
        for (int i = threadIdx.x; i < N; i += T) {
            const int a = i / Q, t = i - a * Q;
            __pipeline_memcpy_async(ta + i, tw_global + 2 * t * a, sizeof(float2));
        }
    }

    // x_j *= W_{2N}^j for j = t + Q q (odd half of a zero-padded forward
    // transform): W_{2N}^t from the table times the constant W_{2P}^q.
    static __device__ __forceinline__ void odd_input(float2 (&v)[P], int t, const float2* tw) {
        const float2 u = tw[t];
#pragma unroll
        for (int q = 1; q < P; ++q) v[q] = cmul(v[q], cmul(u, wpi<P>(q)));
        v[0] = cmul(v[0], u);
    }

    // y_n *= W_{2N}^{-n} for n = a + P b (odd half of a pruned inverse):
    // conj(W_{2N}^a) times the constant conj(W_{2Q}^b).
    static __device__ __forceinline__ void odd_output(float2 (&w)[Q], int a, const float2* tw) {
        const float2 u = cconj(tw[a]);
        w[0] = cmul(w[0], u);
#pragma unroll
        for (int b = 1; b < Q; ++b) w[b] = cmul(w[b], cmul(u, cconj(wpi<Q>(b))));
    }
};

}  // namespace mmk
