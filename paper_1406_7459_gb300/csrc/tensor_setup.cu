// tensor_setup.cu -- one-time FP64 demag tensor and its spectrum.
//
// The paper writes H_demag(i) = sum_l M(l) K(l - i) (Sec. 2, Eq. (7),
// Eqs. (11)-(12)) and takes the FFT of the zero-padded K once, at the start
// (Sec. 3).  The tensor's formula is deferred to the paper's ref. [11]; this
// build uses K = -N with N the cell-to-cell averaged demagnetising tensor of
// two identical rectangular cells (Newell, Williams & Dunlop 1993):
//   |R| <  8 d_max : closed form, the 27-point second difference of Newell's
//                    f (diagonal) and g (off-diagonal) functions;
//   |R| >= 8 d_max : N(R) = V * int T(R+u) prod_a tri_a(u_a) d^3u with the
//                    point-dipole tensor T(s) = (I - 3 s s^T/|s|^2)/(4 pi |s|^3)
//                    and the cell autocorrelation tri_a(u) = (d_a-|u|)/d_a^2,
//                    by Gauss-Legendre on each half-axis: 5 nodes up to
//                    16 d_max, 4 up to 32 d_max, 3 beyond.
// All in FP64 because the closed form cancels catastrophically away from the
// source.  The spectrum of the wrap-padded K is real (each component is even
// or odd on every axis), so it is formed as separable cosine / sine sums
// over the non-negative offsets and stored on the octant kx, ky, kz in
// [0, L/2] in FP32, with the inverse-FFT factor 1/(Lx Ly Lz) folded in.
#include <cmath>

#include "mm_internal.h"

namespace mmk {

struct QuadRules {
    int n[3];
    double s[3][8];            // nodes on [0, 1]
    double w[3][8];            // Gauss-Legendre weight times (1 - s)
    double radius[3];          // upper radius of each tier in units of d_max
};
__constant__ QuadRules c_rules;

constexpr double kNearCells = 8.0;
constexpr double kPi = 3.14159265358979323846;

// Newell's f; terms whose denominator vanishes are zero (their prefactor
// vanishes with it).
__device__ double newell_f(double x, double y, double z) {
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = sqrt(x2 + y2 + z2);
    double out = (2.0 * x2 - y2 - z2) * R / 6.0;
    double d = sqrt(x2 + z2);
    if (d != 0.0) out += 0.5 * y * (z2 - x2) * asinh(y / d);
    d = sqrt(x2 + y2);
    if (d != 0.0) out += 0.5 * z * (y2 - x2) * asinh(z / d);
    d = x * R;
    if (d != 0.0) out += -x * y * z * atan(y * z / d);
    return out;
}

__device__ double newell_g(double x, double y, double z) {
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = sqrt(x2 + y2 + z2);
    double out = -x * y * R / 3.0;
    double d = sqrt(x2 + y2);
    if (d != 0.0) out += x * y * z * asinh(z / d);
    d = sqrt(y2 + z2);
    if (d != 0.0) out += y / 6.0 * (3.0 * z2 - y2) * asinh(x / d);
    d = sqrt(x2 + z2);
    if (d != 0.0) out += x / 6.0 * (3.0 * z2 - x2) * asinh(y / d);
    d = z * R;
    if (d != 0.0) out += -z * z2 / 6.0 * atan(x * y / d);
    d = y * R;
    if (d != 0.0) out += -z * y2 / 2.0 * atan(x * z / d);
    d = x * R;
    if (d != 0.0) out += -z * x2 / 2.0 * atan(y * z / d);
    return out;
}

__device__ void newell_closed(double X, double Y, double Z, double dx, double dy, double dz, double* t) {
    double xx = 0, yy = 0, zz = 0, xy = 0, xz = 0, yz = 0;
    for (int ex = -1; ex <= 1; ++ex)
        for (int ey = -1; ey <= 1; ++ey)
            for (int ez = -1; ez <= 1; ++ez) {
                const double w = (double)((ex == 0 ? 2 : -1) * (ey == 0 ? 2 : -1) * (ez == 0 ? 2 : -1));
                const double a = X + ex * dx, b = Y + ey * dy, c = Z + ez * dz;
                xx += w * newell_f(a, b, c);
                yy += w * newell_f(b, a, c);
                zz += w * newell_f(c, b, a);
                xy += w * newell_g(a, b, c);
                xz += w * newell_g(a, c, b);
                yz += w * newell_g(b, c, a);
            }
    const double s = 1.0 / (4.0 * kPi * dx * dy * dz);
    t[0] = xx * s; t[1] = xy * s; t[2] = xz * s; t[3] = yy * s; t[4] = yz * s; t[5] = zz * s;
}

__device__ void newell_quadrature(double X, double Y, double Z, double dx, double dy, double dz, int tier,
                                  double* t) {
    const int n = c_rules.n[tier];
    double xx = 0, yy = 0, zz = 0, xy = 0, xz = 0, yz = 0;
    for (int a = 0; a < 2 * n; ++a) {
        const int ia = a % n;
        const double sx = X + (a < n ? 1.0 : -1.0) * dx * c_rules.s[tier][ia];
        const double wa = c_rules.w[tier][ia];
        for (int b = 0; b < 2 * n; ++b) {
            const int ib = b % n;
            const double sy = Y + (b < n ? 1.0 : -1.0) * dy * c_rules.s[tier][ib];
            const double wab = wa * c_rules.w[tier][ib];
            for (int c = 0; c < 2 * n; ++c) {
                const int ic = c % n;
                const double sz = Z + (c < n ? 1.0 : -1.0) * dz * c_rules.s[tier][ic];
                const double r2 = sx * sx + sy * sy + sz * sz;
                const double q = wab * c_rules.w[tier][ic] / (r2 * r2 * sqrt(r2));
                xx += (r2 - 3.0 * sx * sx) * q;
                yy += (r2 - 3.0 * sy * sy) * q;
                zz += (r2 - 3.0 * sz * sz) * q;
                xy -= 3.0 * sx * sy * q;
                xz -= 3.0 * sx * sz * q;
                yz -= 3.0 * sy * sz * q;
            }
        }
    }
    const double s = dx * dy * dz / (4.0 * kPi);
    t[0] = xx * s; t[1] = xy * s; t[2] = xz * s; t[3] = yy * s; t[4] = yz * s; t[5] = zz * s;
}

// N on the octant of offsets (i, j, k) >= 0; out[c*count + i + nx*(j + ny*k)].
__global__ void k_tensor_octant(int nx, int ny, int nz, double dx, double dy, double dz, double* __restrict__ out) {
    const size_t count = (size_t)nx * ny * nz;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int i = (int)(t % nx);
    const int j = (int)((t / nx) % ny);
    const int k = (int)(t / ((size_t)nx * ny));
    const double X = __dmul_rn((double)i, dx), Y = __dmul_rn((double)j, dy), Z = __dmul_rn((double)k, dz);
    // tier decision with explicitly rounded operations (no contraction), so
    // that the radius test matches a plain IEEE evaluation
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(X, X), __dmul_rn(Y, Y)), __dmul_rn(Z, Z));
    const double dmax = fmax(dx, fmax(dy, dz));
    double tt[6];
    const double bnear = __dmul_rn(kNearCells, dmax);
    if (r2 < __dmul_rn(bnear, bnear)) {
        newell_closed(X, Y, Z, dx, dy, dz, tt);
    } else {
        int tier = 2;
        for (int q = 0; q < 2; ++q) {
            const double b = __dmul_rn(c_rules.radius[q], dmax);
            if (r2 < __dmul_rn(b, b)) { tier = q; break; }
        }
        newell_quadrature(X, Y, Z, dx, dy, dz, tier, tt);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) out[c * count + t] = tt[c];
}

// component c in (xx, xy, xz, yy, yz, zz) is odd along axis a?
__host__ __device__ inline bool odd_axis(int c, int a) {
    if (a == 0) return c == 1 || c == 2;
    if (a == 1) return c == 1 || c == 4;
    return c == 2 || c == 4;
}

// cs[m] = (cos 2 pi m / L, sin 2 pi m / L), FP64.
__global__ void k_cos_sin(int L, double2* cs) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= L) return;
    double s, c;
    sincospi(2.0 * m / L, &s, &c);
    cs[m] = make_double2(c, s);
}

// Transform along x: in[c][k][j][i], i < nx -> out[c][k][j][kx], kx < Hx.
// Even components: N(0) + 2 sum_{i>0} N(i) cos; odd: 2 sum_{i>0} N(i) sin
// (the factor -i of each odd axis is applied in the last transform).
__global__ void k_tx(int nx, int rows_per_c, int Lx, int Hx, const double* __restrict__ in,
                     double* __restrict__ out, const double2* __restrict__ cs) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)6 * rows_per_c * Hx;
    if (t >= total) return;
    const int kx = (int)(t % Hx);
    const size_t row = t / Hx;
    const int c = (int)(row / rows_per_c);
    const bool odd = odd_axis(c, 0);
    const double* src = in + row * nx;
    double acc = odd ? 0.0 : src[0];
    for (int i = 1; i < nx; ++i) {
        const double2 v = cs[(int)(((long long)kx * i) % Lx)];
        acc += 2.0 * src[i] * (odd ? v.y : v.x);
    }
    out[row * Hx + kx] = acc;
}

// Transform along y: in[c][k][j][kx] (j < ny) -> out[c][k][ky][kx].
__global__ void k_ty(int ny, int nz, int Hx, int Ly, int Hy, const double* __restrict__ in,
                     double* __restrict__ out, const double2* __restrict__ cs) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)6 * nz * Hy * Hx;
    if (t >= total) return;
    const int kx = (int)(t % Hx);
    const int ky = (int)((t / Hx) % Hy);
    const size_t ck = t / ((size_t)Hx * Hy);           // c*nz + k
    const int c = (int)(ck / nz);
    const bool odd = odd_axis(c, 1);
    const double* src = in + ck * (size_t)ny * Hx + kx;
    double acc = odd ? 0.0 : src[0];
    for (int j = 1; j < ny; ++j) {
        const double2 v = cs[(int)(((long long)ky * j) % Ly)];
        acc += 2.0 * src[(size_t)j * Hx] * (odd ? v.y : v.x);
    }
    out[(ck * Hy + ky) * Hx + kx] = acc;
}

// Transform along z and pack: in[c][k][ky][kx] -> Kt[kx][kz][ky][c] (FP32),
// K~ = -(sign) N~ / (Lx Ly Lz), sign = (-i)^2 = -1 for the off-diagonals.
__global__ void k_tz(int nz, int Hx, int Hy, int Lz, int Hz, double scale, const double* __restrict__ in,
                     float* __restrict__ Kt, const double2* __restrict__ cs) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)6 * Hx * Hy * Hz;
    if (t >= total) return;
    const int c = (int)(t % 6);
    const int ky = (int)((t / 6) % Hy);
    const int kz = (int)((t / ((size_t)6 * Hy)) % Hz);
    const int kx = (int)(t / ((size_t)6 * Hy * Hz));
    const bool odd = odd_axis(c, 2);
    const double* src = in + ((size_t)c * nz * Hy + ky) * Hx + kx;
    const size_t kstride = (size_t)Hy * Hx;
    double acc = odd ? 0.0 : src[0];
    for (int k = 1; k < nz; ++k) {
        const double2 v = cs[(int)(((long long)kz * k) % Lz)];
        acc += 2.0 * src[k * kstride] * (odd ? v.y : v.x);
    }
    const bool offdiag = (c == 1 || c == 2 || c == 4);
    Kt[t] = (float)((offdiag ? scale : -scale) * acc);
}

// 2-D (x, y) spectrum per z offset for the direct z sum: with
// N2 = the x and y transforms of N (sine sums for odd axes, without their
// factor -i), the (x, y) DFT of K = -N is -(-i)^(ox+oy) N2.  The kernel
// works with M_z' = i M_z and H_z' = i H_z, which makes every coupling real:
// stored d_c = s_c N2_c / (Lx Ly) with s = (-1, +1, +1, -1, +1, -1) for
// (xx, xy, xz, yy, yz, zz); H_z' takes -d_xz, -d_yz.  Layout
// Kd[kx][dz][c][row], dz = 0..nz-1 (negative offsets: xz, yz change sign),
// each row the even ky then the odd ky, Hyp = Hy rounded up to 4 floats
// (zero tail), so that one kx slice
// is a contiguous run of 16-byte chunks in the order the plane kernel keeps
// it in shared memory.
// With ex.on the exchange operator of Eq. (4) is folded in as the
// zero-padded 7-point stencil (its free-boundary remainder, M(i) times the
// number of missing neighbours / delta^2, is added per cell by the update
// kernel), so that the update needs no neighbour cells.
__global__ void k_pack2d(int nz, int Hx, int Hy, int Hyp, double scale, const double* __restrict__ in,
                         float* __restrict__ Kd, ExchangeFold ex) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)6 * Hx * Hyp * nz;
    if (t >= total) return;
    // a row holds the even ky (0, 2, ..., at positions 0 .. E-1) and then the
    // odd ky (1, 3, ..., at E .. Hy-1), E = (Hy + 1) / 2: the plane kernel's
    // consecutive threads take ky of one parity, so they read consecutive words
    const int pos = (int)(t % Hyp);
    const int c = (int)((t / Hyp) % 6);
    const int dz = (int)((t / ((size_t)6 * Hyp)) % nz);
    const int kx = (int)(t / ((size_t)6 * Hyp * nz));
    const int E = (Hy + 1) / 2;
    if (pos >= Hy) {
        Kd[t] = 0.f;
        return;
    }
    const int ky = pos < E ? 2 * pos : 2 * (pos - E) + 1;
    const double v = in[(((size_t)c * nz + dz) * Hy + ky) * Hx + kx];
    const double sg = (c == 0 || c == 3 || c == 5) ? -1.0 : 1.0;
    double e = 0.0;
    if (ex.on && (c == 0 || c == 3 || c == 5)) {
        // zero-padded 7-point stencil of Eq. (4) in the (kx, ky, dz) domain,
        // axes with a single cell skipped
        if (dz == 0) {
            if (ex.nx > 1) e += (2.0 * cospi(2.0 * kx / ex.Lx) - 2.0) * ex.idx2;
            if (ex.ny > 1) e += (2.0 * cospi(2.0 * ky / ex.Ly) - 2.0) * ex.idy2;
            if (nz > 1) e -= 2.0 * ex.idz2;
        } else if (dz == 1) {
            e += ex.idz2;
        }
        e *= ex.pexch;
    }
    Kd[t] = (float)(scale * (sg * v + e));
}

// Roots and weights of the n-point Gauss-Legendre rule on [-1, 1] by Newton
// iteration on the three-term recurrence of the Legendre polynomials.
static void gauss_legendre(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double p1 = 0, p2 = 0, pp = 0;
        for (int it = 0; it < 100; ++it) {
            p1 = 1.0;
            p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                const double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            const double z1 = z;
            z = z1 - p1 / pp;
            if (std::fabs(z - z1) < 1e-15) break;
        }
        p1 = 1.0;
        p2 = 0.0;
        for (int j = 1; j <= n; ++j) {
            const double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        pp = n * (z * p1 - p2) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

static cudaError_t upload_rules() {
    QuadRules r{};
    const int ns[3] = {5, 4, 3};
    const double radius[3] = {16.0, 32.0, 1e300};
    for (int q = 0; q < 3; ++q) {
        double x[8], w[8];
        gauss_legendre(ns[q], x, w);
        r.n[q] = ns[q];
        r.radius[q] = radius[q];
        for (int i = 0; i < ns[q]; ++i) {
            const double s = 0.5 * (x[i] + 1.0);
            r.s[q][i] = s;
            r.w[q][i] = 0.5 * w[i] * (1.0 - s);
        }
    }
    return cudaMemcpyToSymbol(c_rules, &r, sizeof(r));
}

cudaError_t tensor_octant_fp64(const int grid[3], const double cell[3], double* N_dev, cudaStream_t s) {
    cudaError_t e = upload_rules();
    if (e != cudaSuccess) return e;
    const size_t count = (size_t)grid[0] * grid[1] * grid[2];
    const int T = 128;
    k_tensor_octant<<<(unsigned)((count + T - 1) / T), T, 0, s>>>(grid[0], grid[1], grid[2], cell[0], cell[1],
                                                                  cell[2], N_dev);
    return cudaGetLastError();
}

size_t tensor_work_elems(const int grid[3], const int L[3]) {
    const size_t Hx = L[0] / 2 + 1, Hy = L[1] / 2 + 1;
    const size_t a = (size_t)6 * grid[2] * grid[1] * Hx;       // after x
    const size_t b = (size_t)6 * grid[2] * Hy * Hx;            // after y
    return a > b ? a : b;
}

cudaError_t tensor_spectrum(const int grid[3], const int L[3], const double* N_dev, float* Kt_dev,
                            double* work1, double* work2, cudaStream_t s, float* Kd_dev, ExchangeFold ex,
                            float* Kd0_dev) {
    const int nx = grid[0], ny = grid[1], nz = grid[2];
    const int Hx = L[0] / 2 + 1, Hy = L[1] / 2 + 1, Hz = L[2] / 2 + 1;
    double2* cs = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&cs, sizeof(double2) * (L[0] + L[1] + L[2]), s);
    if (e != cudaSuccess) return e;
    double2 *csx = cs, *csy = cs + L[0], *csz = cs + L[0] + L[1];
    const int T = 256;
    k_cos_sin<<<(L[0] + T - 1) / T, T, 0, s>>>(L[0], csx);
    k_cos_sin<<<(L[1] + T - 1) / T, T, 0, s>>>(L[1], csy);
    k_cos_sin<<<(L[2] + T - 1) / T, T, 0, s>>>(L[2], csz);
    size_t n1 = (size_t)6 * nz * ny * Hx;
    k_tx<<<(unsigned)((n1 + T - 1) / T), T, 0, s>>>(nx, nz * ny, L[0], Hx, N_dev, work1, csx);
    size_t n2 = (size_t)6 * nz * Hy * Hx;
    k_ty<<<(unsigned)((n2 + T - 1) / T), T, 0, s>>>(ny, nz, Hx, L[1], Hy, work1, work2, csy);
    if (Kd_dev) {
        const int Hyp = kd_row(Hy);
        const size_t nd = (size_t)6 * Hx * Hyp * nz;
        k_pack2d<<<(unsigned)((nd + T - 1) / T), T, 0, s>>>(nz, Hx, Hy, Hyp, 1.0 / ((double)L[0] * L[1]), work2,
                                                            Kd_dev, ex);
        if (Kd0_dev)
            k_pack2d<<<(unsigned)((nd + T - 1) / T), T, 0, s>>>(nz, Hx, Hy, Hyp, 1.0 / ((double)L[0] * L[1]), work2,
                                                                Kd0_dev, ExchangeFold{});
    }
    size_t n3 = (size_t)6 * Hx * Hy * Hz;
    const double scale = 1.0 / ((double)L[0] * L[1] * L[2]);
    k_tz<<<(unsigned)((n3 + T - 1) / T), T, 0, s>>>(nz, Hx, Hy, L[2], Hz, scale, work2, Kt_dev, csz);
    e = cudaGetLastError();
    cudaError_t e2 = cudaFreeAsync(cs, s);
    return e != cudaSuccess ? e : e2;
}

// Kt_ex = Kt + the symbol of the zero-padded 7-point exchange stencil of
// Eq. (4) on xx, yy, zz (axes of one cell skipped), in the stored scaling
// 1/(Lx Ly Lz).  The update kernel adds the free-face remainder per cell.
__global__ void k_kt_exchange(Geom g, ExchangeFold ex, double scale, const float* __restrict__ Kt,
                              float* __restrict__ Kt_ex) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)6 * g.Hx * g.Hy * g.Hz;
    if (t >= total) return;
    const int c = (int)(t % 6);
    const int ky = (int)((t / 6) % g.Hy);
    const int kz = (int)((t / ((size_t)6 * g.Hy)) % g.Hz);
    const int kx = (int)(t / ((size_t)6 * g.Hy * g.Hz));
    double e = 0.0;
    if (c == 0 || c == 3 || c == 5) {
        if (g.nx > 1) e += (2.0 * cospi(2.0 * kx / g.Lx) - 2.0) * ex.idx2;
        if (g.ny > 1) e += (2.0 * cospi(2.0 * ky / g.Ly) - 2.0) * ex.idy2;
        if (g.nz > 1) e += (2.0 * cospi(2.0 * kz / g.Lz) - 2.0) * ex.idz2;
        e *= ex.pexch * scale;
    }
    Kt_ex[t] = (float)((double)Kt[t] + e);
}

cudaError_t tensor_fold_exchange3(const Geom& g, ExchangeFold ex, const float* Kt, float* Kt_ex, cudaStream_t s) {
    const size_t n = (size_t)6 * g.Hx * g.Hy * g.Hz;
    const int T = 256;
    k_kt_exchange<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(g, ex, 1.0 / ((double)g.Lx * g.Ly * g.Lz), Kt, Kt_ex);
    return cudaGetLastError();
}

}  // namespace mmk
