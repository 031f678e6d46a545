// Preparation-step kernels (Sec. II.C, Table I upper half): monitoring points,
// Fibonacci integration directions, the harmonic basis, and the FP64
// pseudo-inverse of the fitting matrix by Householder QR.
#include <math.h>

#include <cmath>

#include <vector>

#include "common.cuh"

#include <algorithm>

namespace hsma {

namespace {

constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ void write_target(long long i, double x, double y, double z, double4_32a *o64, float4 *hi,
                                             float4 *lo)
{
    o64[i] = make_double4_32a(x, y, z, 0.0);
    float hx, lx, hy, ly, hz, lz;
    split_f64(x, hx, lx);
    split_f64(y, hy, ly);
    split_f64(z, hz, lz);
    hi[i] = make_float4(hx, hy, hz, 0.f);
    lo[i] = make_float4(lx, ly, lz, 0.f);
}

// Periodic monitoring points (Sec. II.A): Fibonacci latitude grid on the
// circumsphere, x_i for i = 1..K, then the partners x~_i = x_i - k L wrapped
// into the central box (k = nearest integer, ties away from zero).
__global__ void monitor_sphere_kernel(int K, double R0, double Lx, double Ly, double Lz, double4_32a *o64,
                                      float4 *hi, float4 *lo)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    double w = (sqrt(5.0) - 1.0) * 0.5;
    int ii = i + 1;
    double sl = (2.0 * ii - 1.0) / K - 1.0;  // sine of the latitude
    double cl = sqrt(fmax(0.0, 1.0 - sl * sl));
    double az = 2.0 * kPi * ii * w;
    double x = R0 * cl * cos(az), y = R0 * cl * sin(az), z = R0 * sl;
    write_target(i, x, y, z, o64, hi, lo);
    double xt = x - Lx * round(x / Lx);
    double yt = y - Ly * round(y / Ly);
    double zt = z - Lz * round(z / Lz);
    write_target(K + i, xt, yt, zt, o64, hi, lo);
}

// Wall monitoring points for the grounded box: per face f (order -x, +x, -y,
// +y, -z, +z) cnt[f] points of a 2-D golden-ratio lattice
// ((i + 1/2)/n, frac(i w + 1/2)) over the face.
struct FaceCounts {
    int cnt[6];
    int off[6];
};

__global__ void monitor_faces_kernel(FaceCounts fc, int K, double Lx, double Ly, double Lz, double4_32a *o64,
                                     float4 *hi, float4 *lo)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    int f = 0;
    while (f < 5 && i >= fc.off[f] + fc.cnt[f]) ++f;
    int j = i - fc.off[f];
    int n = fc.cnt[f];
    double w = (sqrt(5.0) - 1.0) * 0.5;
    double u = (j + 0.5) / n;
    double v = fmod(j * w + 0.5, 1.0);
    double L[3] = {Lx, Ly, Lz};
    int a = f / 2;
    int ua = (a == 0) ? 1 : 0;
    int va = (a == 2) ? 1 : 2;
    double p[3];
    p[a] = ((f & 1) ? 0.5 : -0.5) * L[a];
    p[ua] = (u - 0.5) * L[ua];
    p[va] = (v - 0.5) * L[va];
    write_target(i, p[0], p[1], p[2], o64, hi, lo);
}

// Fibonacci integration (Sec. II.B): node j = 0..F2 gives the directions
// (theta_j, phi_j) and (theta_j, phi_j + pi) with cos(theta_j) = z_j +
// sin(pi z_j)/pi, z_j = -1 + 2j/F2, phi_j = pi j F1 / F2, both weighted
// (2 pi Rs^2 / F2)(1 + cos(pi z_j)).  Stored as (u_x, u_y, u_z, w).
__global__ void quadrature_kernel(int F2, int F1, double Rs, double4_32a *dirs)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > F2) return;
    double zj = -1.0 + 2.0 * j / F2;
    double ct = fmin(1.0, fmax(-1.0, zj + sin(kPi * zj) / kPi));
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    // phi_j reduced exactly modulo 2 pi: j F1 mod 2 F2 in integer arithmetic
    long long num = ((long long)j * (long long)F1) % (2LL * F2);
    double ph = kPi * (double)num / (double)F2;
    double w = 2.0 * kPi * Rs * Rs / F2 * (1.0 + cos(kPi * zj));
    dirs[2 * j] = make_double4_32a(st * cos(ph), st * sin(ph), ct, w);
    dirs[2 * j + 1] = make_double4_32a(-st * cos(ph), -st * sin(ph), ct, w);
}

// Orthonormal real solid harmonics (|x|/Rs)^n Y_nm by the fully normalised
// Cartesian recurrence: with (x, y, z) scaled by 1/Rs, r2 = x^2 + y^2 + z^2,
// (x + i y)^m = C_m + i S_m and Pbar_n^m = norm(n, m) Pi_n^m, where
// r^n P_n^m(cos theta) e^{i m phi} = Pi_n^m (x + i y)^m and
// norm(n, m) = sqrt((2 - delta_m0)(2n+1)/(4 pi) (n-m)!/(n+m)!),
//   Pbar_m^m = D_m,  Pbar_{m+1}^m = E_m z,
//   Pbar_n^m = a_nm z Pbar_{n-1}^m - b_nm r2 Pbar_{n-2}^m  (n >= m + 2)
// with the coefficients of basis_f64_tables (the plain recurrence
// (n-m) Pi_n^m = (2n-1) z Pi_{n-1}^m - (n+m-1) r2 Pi_{n-2}^m rescaled by the
// norms, so neither (2m-1)!! nor the norm products appear).  Column
// k = n^2 + n + m holds Pbar_n^|m| (C_m for m >= 0, S_|m| for m < 0).
// Layout of the work as in basis_df_kernel below: a warp takes 32
// consecutive points and runs the degree outer, m inner, with the recurrence
// state in shared memory and each degree's row segments stored coalesced from
// a staging tile, so the output's sectors are written once (the m-outer order
// of one thread per row kept every row's sectors partly written until the
// row was done: L2 evicted and re-read them, and capping the rows in flight
// left one block per SM).  Four FP64 operations per recurrence step and one
// per stored value; FP64 issue is slow on this part.
constexpr int kBasisMaxP = 40;
constexpr int kBasisWarps = 2;  // warps per block
static_assert(kBasisMaxP == kBasisTableMaxP, "one coefficient table serves both basis forms");

// The recurrence coefficients of every n, m <= kBasisMaxP in FP64, computed
// once on the host and passed to the kernel by value (no device buffer).
struct BasisF64Tables {
    double a[kBasisMaxP + 1][kBasisMaxP + 1];  // a_nm at [m][n] (n >= m + 2)
    double b[kBasisMaxP + 1][kBasisMaxP + 1];  // b_nm at [m][n]
    double d[kBasisMaxP + 1];                  // D_m
    double e[kBasisMaxP + 1];                  // E_m = sqrt(2m + 3) D_m
};

const BasisF64Tables &basis_f64_tables()
{
    static const BasisF64Tables t = [] {
        BasisF64Tables v{};
        for (int m = 0; m <= kBasisMaxP; ++m) {
            for (int n = m + 2; n <= kBasisMaxP; ++n) {
                const double dn = n, dm = m, q = dn * dn - dm * dm;
                v.a[m][n] = std::sqrt((4.0 * dn * dn - 1.0) / q);
                v.b[m][n] = std::sqrt((2.0 * dn + 1.0) * ((dn - 1.0) * (dn - 1.0) - dm * dm) / ((2.0 * dn - 3.0) * q));
            }
            double d = 1.0 / std::sqrt(4.0 * kPi);
            for (int j = 1; j <= m; ++j) d *= std::sqrt((2.0 * j + 1.0) / (2.0 * j));
            if (m > 0) d *= std::sqrt(2.0);
            v.d[m] = d;
            v.e[m] = std::sqrt(2.0 * m + 3.0) * d;
        }
        return v;
    }();
    return t;
}

__host__ __device__ constexpr size_t basis_smem_bytes(int P, int warps)
{
    // tables a, b ((P+1)^2 each), D, E (P+1 each); per warp: 4 (P+1) state
    // slots x 32 lanes and a 32 x (2P+1) staging tile (8-byte words)
    return 8 * ((size_t)2 * (P + 1) * (P + 1) + (size_t)2 * (P + 1) +
                (size_t)warps * 32 * ((size_t)4 * (P + 1) + (size_t)(2 * P + 1)));
}

__global__ void __launch_bounds__(32 * kBasisWarps) basis_kernel(const __grid_constant__ BasisF64Tables tabs, int P,
                                                                 double inv_rs, long long np,
                                                                 const double *__restrict__ pts, int stride,
                                                                 double *__restrict__ out, int ld)
{
    extern __shared__ double bsm[];
    const int W = P + 1, pitch = 2 * P + 1;
    double *ta = bsm, *tb = bsm + W * W, *td = tb + W * W, *te = td + W;
    for (int t = threadIdx.x; t < W * W; t += blockDim.x) {
        ta[t] = tabs.a[t / W][t % W];
        tb[t] = tabs.b[t / W][t % W];
    }
    for (int m = threadIdx.x; m <= P; m += blockDim.x) {
        td[m] = tabs.d[m];
        te[m] = tabs.e[m];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *wb = te + W + (size_t)warp * 32 * (4 * W + pitch);
    double *pst = wb + lane;  // Pbar at even, then odd degrees; slot m at [32 m]
    double *cs = wb + 64 * W + lane, *ss = wb + 96 * W + lane;
    double *stage = wb + 128 * W;  // [32 rows][pitch]
    const long long ngroups = (np + 31) / 32;
    for (long long g = (long long)blockIdx.x * (blockDim.x >> 5) + warp; g < ngroups;
         g += (long long)gridDim.x * (blockDim.x >> 5)) {
        const long long i0 = g * 32;
        const int rows = (int)min(32LL, np - i0);
        const long long i = i0 + min(lane, rows - 1);  // lanes past the end repeat the last point, unwritten
        const double x = pts[i * stride] * inv_rs, y = pts[i * stride + 1] * inv_rs, z = pts[i * stride + 2] * inv_rs;
        const double r2 = x * x + y * y + z * z;
        double C = 1.0, S = 0.0;  // (x + i y)^n
        double *sc0 = stage + lane * pitch;
        double *og = out + i0 * ld;
        for (int n = 0; n <= P; ++n) {
            double *cur = pst + (n & 1) * 32 * W, *prv = pst + ((n & 1) ^ 1) * 32 * W;
            double *sc = sc0 + n;  // column n + m holds the cosine part, n - m the sine part
            if (n > 0) {
                const double c2 = C * x - S * y;
                S = S * x + C * y;
                C = c2;
            }
            cs[32 * n] = C;
            ss[32 * n] = S;
            cur[32 * n] = td[n];  // m = n
            sc[n] = td[n] * C;
            if (n > 0) {
                sc[-n] = td[n] * S;
                const int m = n - 1;  // m = n - 1
                const double p = te[m] * z;
                cur[32 * m] = p;
                sc[m] = p * cs[32 * m];
                if (m > 0) sc[-m] = p * ss[32 * m];
            }
            const double *an = ta + n, *bn = tb + n;
            for (int m = 0; m + 2 <= n; ++m) {
                const double pn = fma(an[m * W] * z, prv[32 * m], -(bn[m * W] * r2) * cur[32 * m]);
                cur[32 * m] = pn;
                sc[m] = pn * cs[32 * m];
                if (m > 0) sc[-m] = pn * ss[32 * m];
            }
            __syncwarp();
            const int wd = 2 * n + 1, tot = rows * wd;
            const uint32_t cw = ((1u << 20) + (uint32_t)wd - 1u) / (uint32_t)wd;  // ceil(2^20 / (2n + 1))
            double *ob = og + n * n;
#pragma unroll 4
            for (int f = lane; f < tot; f += 32) {
                const int r = (int)(((uint32_t)f * cw) >> 20), j = f - r * wd;
                ob[r * ld + j] = stage[r * pitch + j];
            }
            __syncwarp();
        }
    }
}

// ------------------------------------------- double-float basis evaluation
// Double-float numbers v = hi + lo (two FP32 words, |lo| <= ulp(hi)/2), for
// the basis on the FP32 pipe: GB300 issues FP64 at a small fraction of its
// FP32 rate.  Products follow Dekker's method, the exact error of hi*hi taken
// with one fused multiply-add (TwoProd), the cross terms added to it; both
// products and sums end with Fast2Sum, so every result is a normalised pair.
// Relative error about 2^-46 per operation.
__device__ __forceinline__ float2 df_mul(float2 a, float2 b)
{
    const float p = __fmul_rn(a.x, b.x);
    float e = __fmaf_rn(a.x, b.x, -p);
    e = __fmaf_rn(a.x, b.y, e);
    e = __fmaf_rn(a.y, b.x, e);
    const float s = __fadd_rn(p, e);
    return make_float2(s, __fsub_rn(e, __fsub_rn(s, p)));
}

__device__ __forceinline__ float2 df_sub(float2 a, float2 b)
{
    return df_add_df(a, make_float2(-b.x, -b.y));
}

// a u - b v in one pass: the two leading products and their exact errors
// (TwoProd), TwoSum of the leading products, the errors and the four cross
// terms gathered in FP32, one Fast2Sum.  Same accuracy as two products and a
// difference, in fewer operations.
__device__ __forceinline__ float2 df_dot2_sub(float2 a, float2 u, float2 b, float2 v)
{
    const float p = __fmul_rn(a.x, u.x), q = __fmul_rn(b.x, v.x);
    const float ep = __fmaf_rn(a.x, u.x, -p), eq = __fmaf_rn(b.x, v.x, -q);
    const float s = __fsub_rn(p, q);
    const float bb = __fsub_rn(s, p);
    float e = __fsub_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fadd_rn(q, bb));
    e = __fadd_rn(e, __fsub_rn(ep, eq));
    e = __fmaf_rn(a.x, u.y, e);
    e = __fmaf_rn(a.y, u.x, e);
    e = __fmaf_rn(-b.x, v.y, e);
    e = __fmaf_rn(-b.y, v.x, e);
    const float h = __fadd_rn(s, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ float2 df_of(double v)
{
    float h, l;
    split_f64(v, h, l);
    return make_float2(h, l);
}

// FP64 value of (hi + lo) * 2^k for a normalised pair, assembled in integer
// arithmetic (an FP64 addition of the two words would run on the slow FP64
// pipe).  hi's sign, exponent + k and significand give the FP64 bit pattern
// (kb = (896 + k) << 20 rebiases the exponent field); lo, scaled by an FP32
// power of two to FP64 units of hi's binade and rounded to an integer, is
// added to the pattern's magnitude (negative: subtracted).  A carry out of
// the significand raises the exponent, which is exactly the IEEE layout's
// behaviour; where hi is a power of two and lo points below it the sum lies
// in the binade underneath, whose spacing is half as large, so lo is counted
// in those units.  A hi below 2^-74 (that is, below 2^-74 of the point's
// scale: the kernel scales every point to a largest coordinate in [1, 2))
// gives a signed zero.  kChecked adds the checks for exponent offsets that
// can leave FP64's normal range (result zero below it, infinity above) and
// for a non-finite hi (result NaN); finite points of ordinary size never
// need them.
template <bool kChecked>
__device__ __forceinline__ double df_to_f64_scaled(float2 v, uint32_t kb, int k)
{
    const uint32_t bh = __float_as_uint(v.x), bl = __float_as_uint(v.y);
    const uint32_t sign = bh & 0x80000000u, mag = bh ^ sign;
    const uint32_t eh = mag >> 23;
    const uint32_t down = (uint32_t)((mag & 0x7fffffu) == 0u) & ((bh ^ bl) >> 31);
    // 1 / (FP64 unit of hi's binade) = 2^(179 - eh): FP32 exponent field
    // 306 - eh (<= 254 for eh >= 53), with hi's sign
    const float pw = __uint_as_float(((306u - eh + down) << 23) | sign);
    const int d = __float2int_rn(__fmul_rn(v.y, pw));  // |d| <= 2^28 for a normalised pair
    unsigned long long bits =
        (((unsigned long long)(((mag >> 3) + kb) | sign) << 32) | (unsigned long long)(bh << 29)) +
        (unsigned long long)(long long)d;
    if (eh < 53u) bits = (unsigned long long)sign << 32;
    if (kChecked) {
        const int ed = (int)eh + 896 + k;
        if (ed <= 0) bits = (unsigned long long)sign << 32;
        if (ed >= 2047) bits = (unsigned long long)(sign | 0x7ff00000u) << 32;
        if (eh == 255u) bits = (unsigned long long)(sign | 0x7ff80000u) << 32;
    }
    return __longlong_as_double((long long)bits);
}

// The same orthonormal real solid harmonics as basis_kernel, in double-float
// arithmetic on the FP32 pipe, by the fully normalised form of the recurrence:
// with Pbar_n^m = norm(n, m) Pi_n^m,
//   Pbar_m^m     = D_m,   D_0 = 1/sqrt(4 pi),
//                         D_m = D_{m-1} sqrt((2m+1)/(2m)) (times sqrt 2 at m = 1),
//   Pbar_{m+1}^m = sqrt(2m+3) D_m z,
//   Pbar_n^m     = a_nm z Pbar_{n-1}^m - b_nm r2 Pbar_{n-2}^m,
//     a_nm = sqrt((4n^2 - 1) / (n^2 - m^2)),
//     b_nm = sqrt((2n+1) ((n-1)^2 - m^2) / ((2n-3) (n^2 - m^2))),
// (the ratios norm(n, m) (2n-1) / ((n-m) norm(n-1, m)) and
// norm(n, m) (n+m-1) / ((n-m) norm(n-2, m)) of the unnormalised recurrence),
// so every intermediate stays of order r^n and the norm products disappear.
// Each point is scaled by a power of two 2^-e that brings its largest
// coordinate (over Rs) into [1, 2): a degree-n value is then the double-float
// result times 2^(e n), applied exactly in the FP64 assembly, so small or
// large |x| / Rs cannot leave FP32's exponent range.  The coefficient tables
// are computed once per block in FP64 and kept in shared memory as pairs.
// Accuracy: relative ~1e-14 of the row's scale (r/Rs)^n per value, against
// ~1e-16 for the FP64 kernel.
//
// Layout of the work: a warp takes 32 consecutive points (rows) and runs the
// degree n in the outer loop, m inner, so that each degree completes the
// contiguous row segment [n^2, n^2 + 2n].  The recurrence state of every m
// (Pbar at the last two degrees, in two arrays that alternate with the
// degree's parity, and (x + i y)^m) sits in shared memory, one slot per lane.
// A degree's 2n + 1 values per row go to a shared staging tile; the warp then
// stores the tile's 32 segments with its lanes over consecutive elements of
// the tile (row r = floor(f / (2n + 1)) by a multiply-shift, exact for
// f < 2^20 / (2n + 1)).  Rows are thus written front to back in runs of up
// to 2P + 1 doubles: the 32-byte sectors of a row complete within one or two
// degrees (in the m-outer order every sector of every row in flight stayed
// partly written until the row was done, and L2 evicted and re-read them),
// and each store instruction covers two or three row segments instead of one
// value in each of 32 rows.
//
// The recurrence coefficients do not depend on P: the host computes them once
// in FP64 for every n, m <= 40, splits them into pairs and passes them as a
// kernel parameter; each block copies the (P+1)^2 it needs to shared memory.
constexpr int kBasisDfWarps = 2;  // warps per block

__host__ __device__ constexpr size_t basis_df_smem_bytes(int P, int warps)
{
    // tables a, b ((P+1)^2 each), D, E (P+1 each); per warp: 4 (P+1) state
    // slots x 32 lanes and a 32 x (2P+1) staging tile (8-byte words)
    return 8 * ((size_t)2 * (P + 1) * (P + 1) + (size_t)2 * (P + 1) +
                (size_t)warps * 32 * ((size_t)4 * (P + 1) + (size_t)(2 * P + 1)));
}

struct BasisDfWarp {
    float2 *pst;    // Pbar at even, then odd degrees: slot m of this lane at [32 m]
    float2 *cs;     // (x + i y)^m, real part, slot m at [32 m]
    float2 *ss;     // imaginary part
    double *stage;  // [32 rows][2P + 1]
};

// One group of up to 32 points (rows i0 .. i0 + rows - 1): the degree loop.
template <bool kChecked>
__device__ __forceinline__ void basis_df_rows(int P, const float2 *ta, const float2 *tb, const float2 *td,
                                              const float2 *te, const BasisDfWarp &w, int lane, float2 X,
                                              float2 Y, float2 Z, float2 R2, int e, int rows, double *og,
                                              int ld)
{
    const int W = P + 1, pitch = 2 * P + 1;
    float2 C = make_float2(1.f, 0.f), S = make_float2(0.f, 0.f);  // (x + i y)^n, scaled
    double *srow = w.stage + lane * pitch;
    for (int n = 0; n <= P; ++n) {
        const int en = e * n;
        const uint32_t kb = (uint32_t)(896 + en) << 20;
        float2 *cur = w.pst + (n & 1) * 32 * W, *prv = w.pst + ((n & 1) ^ 1) * 32 * W;
        double *sc = srow + n;  // column n + m holds the cosine part, n - m the sine part
        if (n > 0) {
            const float2 c2 = df_sub(df_mul(C, X), df_mul(S, Y));
            S = df_add_df(df_mul(S, X), df_mul(C, Y));
            C = c2;
        }
        w.cs[32 * n] = C;
        w.ss[32 * n] = S;
        {  // m = n
            const float2 pd = td[n];
            cur[32 * n] = pd;
            sc[n] = df_to_f64_scaled<kChecked>(df_mul(pd, C), kb, en);
            if (n > 0) sc[-n] = df_to_f64_scaled<kChecked>(df_mul(pd, S), kb, en);
        }
        if (n > 0) {  // m = n - 1
            const int m = n - 1;
            const float2 p = df_mul(te[m], Z);
            cur[32 * m] = p;
            if (m == 0) {
                sc[0] = df_to_f64_scaled<kChecked>(p, kb, en);
            } else {
                sc[m] = df_to_f64_scaled<kChecked>(df_mul(p, w.cs[32 * m]), kb, en);
                sc[-m] = df_to_f64_scaled<kChecked>(df_mul(p, w.ss[32 * m]), kb, en);
            }
        }
        if (n >= 2) {  // m = 0: (x + i y)^0 = 1
            const float2 pn = df_dot2_sub(ta[n], df_mul(Z, prv[0]), tb[n], df_mul(R2, cur[0]));
            cur[0] = pn;
            sc[0] = df_to_f64_scaled<kChecked>(pn, kb, en);
        }
        // m >= 1, two orders per pass: their chains are independent, which
        // doubles the instruction-level parallelism of the double-float work
        int m = 1;
        for (; m + 3 <= n; m += 2) {
            const float2 p1a = prv[32 * m], p2a = cur[32 * m], p1b = prv[32 * m + 32], p2b = cur[32 * m + 32];
            const float2 ca = w.cs[32 * m], sa = w.ss[32 * m], cb = w.cs[32 * m + 32], sb = w.ss[32 * m + 32];
            const float2 pa = df_dot2_sub(ta[m * W + n], df_mul(Z, p1a), tb[m * W + n], df_mul(R2, p2a));
            const float2 pb =
                df_dot2_sub(ta[(m + 1) * W + n], df_mul(Z, p1b), tb[(m + 1) * W + n], df_mul(R2, p2b));
            cur[32 * m] = pa;
            cur[32 * m + 32] = pb;
            sc[m] = df_to_f64_scaled<kChecked>(df_mul(pa, ca), kb, en);
            sc[-m] = df_to_f64_scaled<kChecked>(df_mul(pa, sa), kb, en);
            sc[m + 1] = df_to_f64_scaled<kChecked>(df_mul(pb, cb), kb, en);
            sc[-m - 1] = df_to_f64_scaled<kChecked>(df_mul(pb, sb), kb, en);
        }
        if (m + 2 <= n) {
            const float2 p1 = prv[32 * m], p2 = cur[32 * m];
            const float2 pn = df_dot2_sub(ta[m * W + n], df_mul(Z, p1), tb[m * W + n], df_mul(R2, p2));
            cur[32 * m] = pn;
            sc[m] = df_to_f64_scaled<kChecked>(df_mul(pn, w.cs[32 * m]), kb, en);
            sc[-m] = df_to_f64_scaled<kChecked>(df_mul(pn, w.ss[32 * m]), kb, en);
        }
        __syncwarp();
        const int wd = 2 * n + 1, tot = rows * wd;
        const uint32_t cw = ((1u << 20) + (uint32_t)wd - 1u) / (uint32_t)wd;  // ceil(2^20 / (2n + 1))
        double *ob = og + n * n;
#pragma unroll 4
        for (int f = lane; f < tot; f += 32) {
            const int r = (int)(((uint32_t)f * cw) >> 20), j = f - r * wd;
            ob[r * ld + j] = w.stage[r * pitch + j];
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(32 * kBasisDfWarps) basis_df_kernel(const __grid_constant__ BasisDfTables tabs,
                                                                      int P, double inv_rs, long long np,
                                                                      const double *__restrict__ pts, int stride,
                                                                      double *__restrict__ out, long long ld)
{
    extern __shared__ float2 tab[];
    const int W = P + 1, pitch = 2 * P + 1;
    float2 *ta = tab, *tb = tab + W * W, *td = tab + 2 * W * W, *te = td + W;
    for (int t = threadIdx.x; t < W * W; t += blockDim.x) {
        const int m = t / W, n = t % W;
        ta[t] = tabs.a[m][n];
        tb[t] = tabs.b[m][n];
    }
    for (int m = threadIdx.x; m <= P; m += blockDim.x) {
        td[m] = tabs.d[m];
        te[m] = tabs.e[m];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2 *wb = te + W + (size_t)warp * 32 * (4 * W + pitch);
    const BasisDfWarp w{wb + lane, wb + 64 * W + lane, wb + 96 * W + lane, reinterpret_cast<double *>(wb + 128 * W)};
    const long long ngroups = (np + 31) / 32;
    for (long long g = (long long)blockIdx.x * (blockDim.x >> 5) + warp; g < ngroups;
         g += (long long)gridDim.x * (blockDim.x >> 5)) {
        const long long i0 = g * 32;
        const int rows = (int)min(32LL, np - i0);
        const long long i = i0 + min(lane, rows - 1);  // lanes past the end repeat the last point, unwritten
        const double px = pts[i * stride], py = pts[i * stride + 1], pz = pts[i * stride + 2];
        const double big = fmax(fabs(px), fmax(fabs(py), fabs(pz))) * inv_rs;
        const int eb = min((__double2hiint(big) >> 20) & 0x7ff, 2045);  // biased exponent of the largest
        int e = 0;
        double f = 0.0;  // a point at the origin (or below FP64's normal range) is the origin
        if (eb > 0) {
            e = eb - 1023;
            f = inv_rs * __hiloint2double((2046 - eb) << 20, 0);  // inv_rs 2^-e
        }
        const float2 X = df_of(px * f), Y = df_of(py * f), Z = df_of(pz * f);
        const float2 R2 = df_add_df(df_add_df(df_mul(X, X), df_mul(Y, Y)), df_mul(Z, Z));
        // exponent offsets e n with n <= P stay inside FP64's range for every
        // value of FP32 size, and a finite point gives finite values
        const bool finite = isfinite(px) && isfinite(py) && isfinite(pz);
        const bool plain = __all_sync(0xffffffffu, finite && abs(e) * P <= 895);
        if (plain)
            basis_df_rows<false>(P, ta, tb, td, te, w, lane, X, Y, Z, R2, e, rows, out + i0 * ld, (int)ld);
        else
            basis_df_rows<true>(P, ta, tb, td, te, w, lane, X, Y, Z, R2, e, rows, out + i0 * ld, (int)ld);
    }
}

// Fitting matrix: periodic  M_ik = B_{k+1}(x_i) - B_{k+1}(x~_i)  (column 0
// dropped, it is identically zero); grounded M_ik = B_k(x_i).  Written both
// column-major (for the QR) and row-major (for the refinement residual).
__global__ void fitting_matrix_kernel(int K, int Nb, int ncols, int drop, const double *Bx, const double *Bxt,
                                      double *Mcol, double *Mrow)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)K * ncols) return;
    int i = (int)(t / ncols), c = (int)(t % ncols);
    int k = c + drop;
    double v = Bx[(long long)i * Nb + k];
    if (Bxt) v -= Bxt[(long long)i * Nb + k];
    Mrow[t] = v;
    Mcol[(long long)c * K + i] = v;
}

// ---------------------------------------------------------------- QR
// Column equilibration: scale[c] = 1/||W(:,c)||, W(:,c) *= scale[c].
__global__ void equilibrate_kernel(double *W, int K, double *scale, int *rank_ok)
{
    __shared__ double red[32];
    int c = blockIdx.x;
    double *col = W + (long long)c * K;
    double s = 0.0;
    for (int i = threadIdx.x; i < K; i += blockDim.x) s += col[i] * col[i];
    s = block_sum(s, red);
    double sc = (s > 0.0) ? 1.0 / sqrt(s) : 0.0;
    if (s == 0.0 && threadIdx.x == 0) *rank_ok = 0;
    for (int i = threadIdx.x; i < K; i += blockDim.x) col[i] *= sc;
    if (threadIdx.x == 0) scale[c] = sc;
}

// Householder step j (Golub & Van Loan, Alg. 5.2.1 in spirit): block 0
// records the reflector v = W(j:,j) - alpha e_1 (its top entry vtop, its
// squared norm vv and R_jj = alpha); block b >= 1 applies the reflector to
// column j + b.  Column j itself is not modified in this launch.
__global__ void qr_step_kernel(double *W, int K, int n, int j, double *vtop, double *vv, double *diag,
                               int *rank_ok)
{
    __shared__ double red[32];
    const double *cj = W + (long long)j * K;
    double below = 0.0;
    for (int i = j + 1 + threadIdx.x; i < K; i += blockDim.x) below += cj[i] * cj[i];
    below = block_sum(below, red);
    double a = cj[j];
    double nrm = sqrt(below + a * a);
    double alpha = (a > 0.0) ? -nrm : nrm;
    double v0 = a - alpha;
    double vvj = below + v0 * v0;
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) {
            vtop[j] = v0;
            vv[j] = vvj;
            diag[j] = alpha;
            if (!(nrm > 0.0)) *rank_ok = 0;
        }
        return;
    }
    if (!(vvj > 0.0)) return;
    int c = j + blockIdx.x;
    if (c >= n) return;
    double *cc = W + (long long)c * K;
    double d = 0.0;
    for (int i = j + 1 + threadIdx.x; i < K; i += blockDim.x) d += cj[i] * cc[i];
    d = block_sum(d, red);
    d += v0 * cc[j];
    double tau = 2.0 * d / vvj;
    if (threadIdx.x == 0) cc[j] -= tau * v0;
    for (int i = j + 1 + threadIdx.x; i < K; i += blockDim.x) cc[i] -= tau * cj[i];
}

// Column c of Q_1 = H_0 H_1 ... H_{n-1} [I_n; 0]: start from e_c and apply the
// reflectors from the last to the first.  The K-vector lives in shared memory.
__global__ void qr_form_q_kernel(const double *W, int K, int n, const double *vtop, const double *vv,
                                 double *Q1 /* K x n column-major */)
{
    extern __shared__ double y[];
    __shared__ double red[32];
    int c = blockIdx.x;
    for (int i = threadIdx.x; i < K; i += blockDim.x) y[i] = (i == c) ? 1.0 : 0.0;
    __syncthreads();
    for (int j = n - 1; j >= 0; --j) {
        const double *cj = W + (long long)j * K;
        double d = 0.0;
        for (int i = j + 1 + threadIdx.x; i < K; i += blockDim.x) d += cj[i] * y[i];
        d = block_sum(d, red);
        d += vtop[j] * y[j];
        double tau = (vv[j] > 0.0) ? 2.0 * d / vv[j] : 0.0;
        __syncthreads();
        if (threadIdx.x == 0) y[j] -= tau * vtop[j];
        for (int i = j + 1 + threadIdx.x; i < K; i += blockDim.x) y[i] -= tau * cj[i];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < K; i += blockDim.x) Q1[(long long)c * K + i] = y[i];
}

// Column c of R^{-1} by back substitution (R upper triangular: strict upper
// part in W above the diagonal, diagonal in diag).  x lives in shared memory.
__global__ void r_inverse_kernel(const double *W, int K, int n, const double *diag, double *Rinv /* n x n row-major */)
{
    extern __shared__ double x[];
    __shared__ double red[32];
    int c = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) x[c] = 1.0 / diag[c];
    __syncthreads();
    for (int i = c - 1; i >= 0; --i) {
        double s = 0.0;
        for (int k = i + 1 + threadIdx.x; k <= c; k += blockDim.x) s += W[(long long)k * K + i] * x[k];
        s = block_sum(s, red);
        if (threadIdx.x == 0) x[i] = -s / diag[i];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) Rinv[(long long)i * n + c] = x[i];
}

// M+ = S R^{-1} Q_1^T, row-major n x K:  Mp[k][i] = scale[k] sum_c Rinv[k][c] Q1[i][c].
__global__ void pinv_gemm_kernel(int K, int n, const double *Rinv, const double *Q1, const double *scale,
                                 double *Mp)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * K) return;
    int k = (int)(t / K), i = (int)(t % K);
    double s = 0.0;
    for (int c = k; c < n; ++c) s += Rinv[(long long)k * n + c] * Q1[(long long)c * K + i];
    Mp[t] = scale[k] * s;
}

__global__ void cond_kernel(const double *diag, int n, double *cond)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lo = INFINITY, hi = 0.0;
    for (int j = 0; j < n; ++j) {
        double a = fabs(diag[j]);
        lo = fmin(lo, a);
        hi = fmax(hi, a);
    }
    *cond = (lo > 0.0) ? hi / lo : INFINITY;
}

}  // namespace

int launch_monitor_sphere(int K, double R0, const double L[3], double4_32a *o64, float4 *hi, float4 *lo, cudaStream_t st)
{
    monitor_sphere_kernel<<<(K + 127) / 128, 128, 0, st>>>(K, R0, L[0], L[1], L[2], o64, hi, lo);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

int launch_monitor_faces(const int cnt[6], const double L[3], double4_32a *o64, float4 *hi, float4 *lo, cudaStream_t st)
{
    FaceCounts fc;
    int off = 0;
    for (int f = 0; f < 6; ++f) {
        fc.cnt[f] = cnt[f];
        fc.off[f] = off;
        off += cnt[f];
    }
    monitor_faces_kernel<<<(off + 127) / 128, 128, 0, st>>>(fc, off, L[0], L[1], L[2], o64, hi, lo);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

const BasisDfTables &basis_df_tables()
{
    static const BasisDfTables t = [] {
        const BasisF64Tables &f = basis_f64_tables();
        BasisDfTables v{};
        auto pair = [](double x) {
            const float h = (float)x;
            return make_float2(h, (float)(x - (double)h));
        };
        for (int m = 0; m <= kBasisTableMaxP; ++m) {
            for (int n = 0; n <= kBasisTableMaxP; ++n) {
                v.a[m][n] = pair(f.a[m][n]);
                v.b[m][n] = pair(f.b[m][n]);
            }
            v.d[m] = pair(f.d[m]);
            v.e[m] = pair(f.e[m]);
        }
        return v;
    }();
    return t;
}

double basis_norm(int n, int m)
{
    // sqrt((2 - delta_m0)(2n+1)/(4 pi) (n-m)!/(n+m)!), m >= 0
    double r = 1.0;
    for (int t = n - m + 1; t <= n + m; ++t) r /= (double)t;
    return std::sqrt((m == 0 ? 1.0 : 2.0) * (2.0 * n + 1.0) / (4.0 * kPi) * r);
}

int launch_quadrature(int F2, int F1, double Rs, double4_32a *dirs, cudaStream_t st)
{
    quadrature_kernel<<<(F2 + 1 + 127) / 128, 128, 0, st>>>(F2, F1, Rs, dirs);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

int launch_basis(int P, double Rs, long long np, const double *pts, int stride, double *out, long long ld,
                 cudaStream_t st)
{
    if (np <= 0) return HSMA_OK;
    // the kernel indexes a group's 32 rows with 32-bit offsets r ld + column
    if (P < 0 || P > kBasisMaxP || ld < (long long)(P + 1) * (P + 1) || ld > (1LL << 26)) return HSMA_E_ARG;
    int dev = 0, sms = 1, per_sm = 0;
    HSMA_CUDA_TRY(cudaGetDevice(&dev));
    HSMA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = basis_smem_bytes(P, kBasisWarps);
    HSMA_CUDA_TRY(cudaFuncSetAttribute(basis_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    HSMA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, basis_kernel, 32 * kBasisWarps, smem));
    if (per_sm < 1) return HSMA_E_ARG;
    const long long groups = (np + 31) / 32;
    const long long blocks = std::min<long long>((groups + kBasisWarps - 1) / kBasisWarps, (long long)sms * per_sm);
    basis_kernel<<<(unsigned)blocks, 32 * kBasisWarps, smem, st>>>(basis_f64_tables(), P, 1.0 / Rs, np, pts, stride,
                                                                   out, (int)ld);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

int launch_basis_df(int P, double Rs, long long np, const double *pts, int stride, double *out, long long ld,
                    cudaStream_t st)
{
    if (np <= 0) return HSMA_OK;
    // the kernel indexes a group's 32 rows with 32-bit offsets r ld + column
    if (P < 0 || P > kBasisMaxP || ld < (long long)(P + 1) * (P + 1) || ld > (1LL << 26)) return HSMA_E_ARG;
    int dev = 0, sms = 1, per_sm = 0;
    HSMA_CUDA_TRY(cudaGetDevice(&dev));
    HSMA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = basis_df_smem_bytes(P, kBasisDfWarps);
    HSMA_CUDA_TRY(cudaFuncSetAttribute(basis_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    HSMA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, basis_df_kernel, 32 * kBasisDfWarps, smem));
    if (per_sm < 1) return HSMA_E_ARG;
    const long long groups = (np + 31) / 32;
    const long long blocks =
        std::min<long long>((groups + kBasisDfWarps - 1) / kBasisDfWarps, (long long)sms * per_sm);
    basis_df_kernel<<<(unsigned)blocks, 32 * kBasisDfWarps, smem, st>>>(basis_df_tables(), P, 1.0 / Rs, np, pts,
                                                                       stride, out, ld);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

int launch_fitting_matrix(int K, int Nb, int ncols, int drop, const double *Bx, const double *Bxt, double *Mcol,
                          double *Mrow, cudaStream_t st)
{
    long long tot = (long long)K * ncols;
    fitting_matrix_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(K, Nb, ncols, drop, Bx, Bxt, Mcol, Mrow);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

// Pseudo-inverse of the K x n matrix held column-major in Wcol (destroyed):
// Mp (n x K row-major) = S R^{-1} Q_1^T of the column-equilibrated matrix.
int build_pseudo_inverse(int K, int n, double *Wcol, double *Mp, double *cond_host, int *rank_ok_host,
                         cudaStream_t st)
{
    double *scale = nullptr, *vtop = nullptr, *vv = nullptr, *diag = nullptr, *Q1 = nullptr, *Rinv = nullptr,
           *cond = nullptr;
    int *rank_ok = nullptr;
    // the temporaries are freed on every return path (cudaFree waits for the
    // device work that uses them)
    struct Temporaries {
        void **p[4];
        ~Temporaries()
        {
            for (void **q : p)
                if (*q) dev_free(*q);
        }
    } temps{{(void **)&scale, (void **)&rank_ok, (void **)&Q1, (void **)&Rinv}};
    size_t nd = (size_t)n;
    HSMA_CUDA_TRY(dev_malloc(&scale, nd * 4 * sizeof(double) + sizeof(double) + 16));
    vtop = scale + nd;
    vv = vtop + nd;
    diag = vv + nd;
    cond = diag + nd;
    HSMA_CUDA_TRY(dev_malloc(&rank_ok, sizeof(int)));
    HSMA_CUDA_TRY(dev_malloc(&Q1, (size_t)K * n * sizeof(double)));
    HSMA_CUDA_TRY(dev_malloc(&Rinv, (size_t)n * n * sizeof(double)));
    int one = 1;
    HSMA_CUDA_TRY(cudaMemcpyAsync(rank_ok, &one, sizeof(int), cudaMemcpyHostToDevice, st));
    equilibrate_kernel<<<n, 256, 0, st>>>(Wcol, K, scale, rank_ok);
    HSMA_LAUNCHED();
    for (int j = 0; j < n; ++j) {
        qr_step_kernel<<<n - j, 256, 0, st>>>(Wcol, K, n, j, vtop, vv, diag, rank_ok);
        HSMA_LAUNCHED();
    }
    size_t smq = (size_t)K * sizeof(double);
    HSMA_CUDA_TRY(cudaFuncSetAttribute(qr_form_q_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smq));
    qr_form_q_kernel<<<n, 256, smq, st>>>(Wcol, K, n, vtop, vv, Q1);
    HSMA_LAUNCHED();
    size_t smr = (size_t)n * sizeof(double);
    HSMA_CUDA_TRY(cudaFuncSetAttribute(r_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr));
    r_inverse_kernel<<<n, 128, smr, st>>>(Wcol, K, n, diag, Rinv);
    HSMA_LAUNCHED();
    long long tot = (long long)n * K;
    pinv_gemm_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(K, n, Rinv, Q1, scale, Mp);
    HSMA_LAUNCHED();
    cond_kernel<<<1, 32, 0, st>>>(diag, n, cond);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    HSMA_CUDA_TRY(cudaMemcpyAsync(cond_host, cond, sizeof(double), cudaMemcpyDeviceToHost, st));
    HSMA_CUDA_TRY(cudaMemcpyAsync(rank_ok_host, rank_ok, sizeof(int), cudaMemcpyDeviceToHost, st));
    HSMA_CUDA_TRY(cudaStreamSynchronize(st));
    return HSMA_OK;
}

}  // namespace hsma
