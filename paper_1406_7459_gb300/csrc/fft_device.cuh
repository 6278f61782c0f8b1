// fft_device.cuh -- FP32 complex FFT building blocks for the demag passes.
//
// The demag field is a zero-padded discrete convolution evaluated with FFTs
// (Sec. 2, Eqs. (8)-(10); Sec. 3, Eqs. (14)-(16)).  The paper used a
// single-precision library FFT; this file is the project's own.
//
// Design: a batch of lines sits in shared memory; each radix-R stage of a
// Stockham (self-sorting) transform has every thread take butterflies in
// turn: load R inputs into registers, apply the stage twiddles and a radix-R
// DFT, store the R outputs into the other buffer of a ping-pong pair.  The
// result comes out in natural order with no bit reversal.  Radices 2, 3, 4, 5, 8, 16 cover every
// 2^a 3^b 5^c length.  Forward transforms use W = exp(-2 pi i / L); the
// inverse is conj(FFT(conj(x))), unnormalised (the 1/(Lx Ly Lz) factor is
// folded into the stored tensor spectrum).
//
// Shared-memory lines are padded by one element every 16 (padi) so that the
// strided butterfly stores of the early stages do not pile onto two banks.
#pragma once
#include <cuda_runtime.h>

namespace mmk {

constexpr int kMaxStages = 12;

struct AxisPlan {
    int L;                    // transform length (1 = identity)
    int nst;                  // number of stages
    int rad[kMaxStages];      // radix of each stage, in execution order
};

__host__ __device__ __forceinline__ int padi(int e) { return e + (e >> 4); }

// x / d as a multiply-high by ceil(2^32 / d): exact for 0 <= x, d < 2^16
// (the error term x (ceil(2^32/d) d - 2^32) / 2^32 stays below 1 / d).
struct FastDiv {
    unsigned m;
    int d;
    __device__ __forceinline__ explicit FastDiv(int d_) : m(d_ > 1 ? 0xFFFFFFFFu / (unsigned)d_ + 1u : 0u), d(d_) {}
    __device__ __forceinline__ int div(int x) const { return d > 1 ? (int)__umulhi((unsigned)x, m) : x; }
};

// The block-strided flat index t = threadIdx.x + i blockDim.x as t = q d + r,
// advanced by next() without a division per step (any t).
struct StrideDiv {
    int q, r, dq, dr, d;
    __device__ __forceinline__ explicit StrideDiv(int d_) : d(d_) {
        q = (int)threadIdx.x / d_;
        r = (int)threadIdx.x - q * d_;
        dq = (int)blockDim.x / d_;
        dr = (int)blockDim.x - dq * d_;
    }
    __device__ __forceinline__ void next() {
        r += dr;
        q += dq;
        if (r >= d) {
            r -= d;
            ++q;
        }
    }
};
__host__ __device__ __forceinline__ int padded_len(int L) { return L + (L >> 4) + 1; }

// Complex add / subtract as one packed two-lane FP32 instruction (Blackwell
// f32x2; each lane is an ordinary IEEE round-to-nearest add, so results are
// identical to two scalar adds).
__device__ __forceinline__ unsigned long long f2_pack(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
}
// acc + s * a for a real s and complex a (packed FMA with s in both lanes)
__device__ __forceinline__ float2 cfma_real(float s, float2 a, float2 acc) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_pack(make_float2(s, s))), "l"(f2_pack(a)), "l"(f2_pack(acc)));
    return f2_unpack(r);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }   // a * (-i)
__device__ __forceinline__ float2 mul_pi(float2 a) { return make_float2(-a.y, a.x); }   // a * (+i)

// Mathematical constants of the small DFTs.
constexpr float kSqrtHalf = 0.70710678118654752440f;   // cos(pi/4)
constexpr float kCos8 = 0.92387953251128675613f;       // cos(pi/8)
constexpr float kSin8 = 0.38268343236508977173f;       // sin(pi/8)
constexpr float kSqrt3Half = 0.86602540378443864676f;  // sin(2 pi/3)
constexpr float kC51 = 0.30901699437494742410f;        // cos(2 pi/5)
constexpr float kC52 = -0.80901699437494742410f;       // cos(4 pi/5)
constexpr float kS51 = 0.95105651629515357212f;        // sin(2 pi/5)
constexpr float kS52 = 0.58778525229247312917f;        // sin(4 pi/5)

// ---- forward radix-R DFTs in registers: b_q = sum_r a_r W_R^{r q} -------

__device__ __forceinline__ void dft2(float2* a) {
    float2 t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
}

__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
    float2 t2 = cadd(a1, a3), t3 = mul_mi(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

__device__ __forceinline__ void dft4(float2* a) { dft4(a[0], a[1], a[2], a[3]); }

__device__ __forceinline__ void dft8(float2* a) {
    float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
    float2 o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
    dft4(e0, e1, e2, e3);
    dft4(o0, o1, o2, o3);
    // o_q *= W_8^q
    o1 = make_float2(kSqrtHalf * (o1.x + o1.y), kSqrtHalf * (o1.y - o1.x));
    o2 = mul_mi(o2);
    o3 = make_float2(kSqrtHalf * (o3.y - o3.x), -kSqrtHalf * (o3.x + o3.y));
    a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
    a[1] = cadd(e1, o1); a[5] = csub(e1, o1);
    a[2] = cadd(e2, o2); a[6] = csub(e2, o2);
    a[3] = cadd(e3, o3); a[7] = csub(e3, o3);
}

__device__ __forceinline__ void dft16(float2* a) {
    // 4 x 4: columns (stride 4) first, twiddle W_16^{r q}, then rows.
    float2 c[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        c[r][0] = a[r]; c[r][1] = a[r + 4]; c[r][2] = a[r + 8]; c[r][3] = a[r + 12];
        dft4(c[r][0], c[r][1], c[r][2], c[r][3]);
    }
    // twiddles W_16^{r q}: r = input column, q = output of the first DFT4
    const float2 w1 = make_float2(kCos8, -kSin8);
    const float2 w2 = make_float2(kSqrtHalf, -kSqrtHalf);
    const float2 w3 = make_float2(kSin8, -kCos8);
    const float2 w6 = make_float2(-kSqrtHalf, -kSqrtHalf);
    const float2 w9 = make_float2(-kCos8, kSin8);
    c[1][1] = cmul(c[1][1], w1); c[1][2] = cmul(c[1][2], w2); c[1][3] = cmul(c[1][3], w3);
    c[2][1] = cmul(c[2][1], w2); c[2][2] = mul_mi(c[2][2]);   c[2][3] = cmul(c[2][3], w6);
    c[3][1] = cmul(c[3][1], w3); c[3][2] = cmul(c[3][2], w6); c[3][3] = cmul(c[3][3], w9);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float2 x0 = c[0][q], x1 = c[1][q], x2 = c[2][q], x3 = c[3][q];
        dft4(x0, x1, x2, x3);
        a[q] = x0; a[q + 4] = x1; a[q + 8] = x2; a[q + 12] = x3;
    }
}

__device__ __forceinline__ void dft3(float2* a) {
    float2 t = cadd(a[1], a[2]);
    float2 u = csub(a[1], a[2]);
    float2 m = make_float2(a[0].x - 0.5f * t.x, a[0].y - 0.5f * t.y);
    a[0] = cadd(a[0], t);
    float2 su = mul_mi(cscale(u, kSqrt3Half));     // -i (sqrt3/2) u
    a[1] = cadd(m, su);
    a[2] = csub(m, su);
}

__device__ __forceinline__ void dft5(float2* a) {
    float2 t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
    float2 u1 = csub(a[1], a[4]), u2 = csub(a[2], a[3]);
    float2 m1 = make_float2(a[0].x + kC51 * t1.x + kC52 * t2.x, a[0].y + kC51 * t1.y + kC52 * t2.y);
    float2 m2 = make_float2(a[0].x + kC52 * t1.x + kC51 * t2.x, a[0].y + kC52 * t1.y + kC51 * t2.y);
    float2 n1 = make_float2(kS51 * u1.x + kS52 * u2.x, kS51 * u1.y + kS52 * u2.y);
    float2 n2 = make_float2(kS52 * u1.x - kS51 * u2.x, kS52 * u1.y - kS51 * u2.y);
    a[0] = cadd(a[0], cadd(t1, t2));
    a[1] = cadd(m1, mul_mi(n1));
    a[4] = cadd(m1, mul_pi(n1));
    a[2] = cadd(m2, mul_mi(n2));
    a[3] = cadd(m2, mul_pi(n2));
}

template <int R> __device__ __forceinline__ void dft(float2* a);
template <> __device__ __forceinline__ void dft<2>(float2* a) { dft2(a); }
template <> __device__ __forceinline__ void dft<3>(float2* a) { dft3(a); }
template <> __device__ __forceinline__ void dft<4>(float2* a) { dft4(a); }
template <> __device__ __forceinline__ void dft<5>(float2* a) { dft5(a); }
template <> __device__ __forceinline__ void dft<8>(float2* a) { dft8(a); }
template <> __device__ __forceinline__ void dft<16>(float2* a) { dft16(a); }

// One Stockham stage from src to dst over `nlines` lines (line l of a
// buffer starts at base + l*lstride, element e at padi(e)).  Ns = product of
// the radices already applied.  Inputs with index >= n_in are taken as zero
// (pruned, zero-padded input) and never read.  conj_in / conj_out implement
// the inverse transform on the first / last stage.  Every thread of the
// block must enter; ends with a barrier.
template <int R>
__device__ __forceinline__ void stockham_stage(const float2* src, float2* dst, int lstride, int nlines, int L,
                                               int Ns, const float2* __restrict__ tw, int n_in, bool conj_in,
                                               bool conj_out) {
    const int nb = L / R;
    const int total = nb * nlines;
    const int tstride = L / (Ns * R);
    // (line, j) of work item g = line nb + j advanced without a division per
    // item; j / Ns by multiply-high (j, Ns < kMaxLen <= 2^16)
    const FastDiv byNs(Ns);
    StrideDiv w(nb);
    for (int g = threadIdx.x; g < total; g += blockDim.x, w.next()) {
        const int line = w.q, j = w.r;
        const int jq = byNs.div(j);                           // j / Ns
        const int k = j - jq * Ns;
        const float2* p = src + line * lstride;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int e = j + r * nb;
            float2 a = (e < n_in) ? p[padi(e)] : make_float2(0.f, 0.f);
            if (conj_in) a.y = -a.y;
            if (r > 0 && k > 0) a = cmul(a, __ldg(tw + r * k * tstride));
            v[r] = a;
        }
        dft<R>(v);
        float2* q = dst + line * lstride;
        const int o = jq * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float2 a = v[r];
            if (conj_out) a.y = -a.y;
            q[padi(o + r * Ns)] = a;
        }
    }
    __syncthreads();
}

// In-place transform of `nlines` lines of length P.L held in shared memory
// at buf (line stride lstride), using `scratch` (room for `group` lines of
// the same stride) as the other half of the Stockham ping-pong.  Lines are
// processed `group` at a time.  With an odd number of stages the group is
// first copied to scratch so that the last stage lands back in buf.
// Starts and ends with a barrier.
__device__ __forceinline__ void fft_lines(float2* buf, float2* scratch, int lstride, int nlines, int group,
                                          const AxisPlan& P, const float2* __restrict__ tw, int n_in,
                                          bool inverse) {
    __syncthreads();
    if (P.nst == 0) return;
    for (int g0 = 0; g0 < nlines; g0 += group) {
        const int nl = min(group, nlines - g0);
        float2* a = buf + g0 * lstride;
        const float2* src = a;
        float2* dst = scratch;
        if (P.nst & 1) {
            StrideDiv w(n_in);
            for (int t = threadIdx.x; t < nl * n_in; t += blockDim.x, w.next())
                scratch[w.q * lstride + padi(w.r)] = a[w.q * lstride + padi(w.r)];
            __syncthreads();
            src = scratch;
            dst = a;
        }
        int Ns = 1;
        for (int s = 0; s < P.nst; ++s) {
            const int R = P.rad[s];
            const bool ci = inverse && s == 0;
            const bool co = inverse && s == P.nst - 1;
            const int nin = (s == 0) ? n_in : P.L;
            switch (R) {
                case 2: stockham_stage<2>(src, dst, lstride, nl, P.L, Ns, tw, nin, ci, co); break;
                case 3: stockham_stage<3>(src, dst, lstride, nl, P.L, Ns, tw, nin, ci, co); break;
                case 4: stockham_stage<4>(src, dst, lstride, nl, P.L, Ns, tw, nin, ci, co); break;
                case 5: stockham_stage<5>(src, dst, lstride, nl, P.L, Ns, tw, nin, ci, co); break;
                case 8: stockham_stage<8>(src, dst, lstride, nl, P.L, Ns, tw, nin, ci, co); break;
                default: stockham_stage<16>(src, dst, lstride, nl, P.L, Ns, tw, nin, ci, co); break;
            }
            Ns *= R;
            float2* t = const_cast<float2*>(src);
            src = dst;
            dst = t;
        }
    }
}

}  // namespace mmk
