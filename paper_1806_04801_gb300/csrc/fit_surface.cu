// Fit, harmonic surface mapping and energy/forces (Sec. II.A-C).
//
//  fit_fp64          b from the monitoring potentials (periodic:
//                    b_i = Phi_in(x~_i) - Phi_in(x_i); grounded: b_i = -Phi_in(x_i))
//                    and A = M+ b (FP64 matrix-vector product per system).
//  surface_charges   at each integration direction u_j: Phi_out(Rs u_j) and
//                    sigma(Rs u_j) = (1/Rs) sum n A_nm B_nm(Rs u_j); the point
//                    images carry Q_sigma = w sigma/(4 pi) at Rs u_j and the
//                    dipole pair +-p/dr, p = w Phi_out/(4 pi), at (Rs -+ dr/2) u_j
//                    (Eqs. "green", "cd", "integrals" and the Fibonacci rule).
//  surface_pairs     potential and field of those images at every particle.
//  finalize          U = 1/2 sum q_i (Phi_in + Phi_out), F_i = q_i E_i.
#include <math.h>

#include "common.cuh"

namespace hsma {

namespace {

constexpr double kPi = 3.14159265358979323846;

__global__ void fit_fp64_kernel(const SysDesc *sys, int bc, int K, int ncols, int Nb, const double *Mp,
                                const double *phi_tgt, const int *mon_inv, double *b_out, double *A)
{
    const SysDesc sd = sys[blockIdx.y];
    const double *ph = phi_tgt + sd.tgt_off + sd.n;  // monitoring targets
    const int drop = (bc == HSMA_BC_PERIODIC) ? 1 : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * (blockDim.x >> 5) + warp;
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < K; i += blockDim.x)
            b_out[(long long)blockIdx.y * K + i] = rhs_at(ph, mon_inv, K, i, drop != 0);
        if (drop && threadIdx.x == 0) A[(long long)blockIdx.y * Nb] = 0.0;
    }
    if (c >= ncols) return;
    const double *row = Mp + (long long)c * K;
    double s = 0.0;
    for (int i = lane; i < K; i += 32) s += row[i] * rhs_at(ph, mon_inv, K, i, drop != 0);
    s = warp_sum(s);
    if (lane == 0) A[(long long)blockIdx.y * Nb + c + drop] = s;
}

__device__ __forceinline__ int degree_of(int k)
{
    int n = (int)sqrt((double)k);
    while (n * n > k) --n;
    while ((n + 1) * (n + 1) <= k) ++n;
    return n;
}

// One warp per (system, direction).
__global__ void surface_charges_kernel(int ndir, int Nb, const double *Bq, const double4_32a *dirs, const double *A,
                                       double Rs, double2 *img)
{
    const int lane = threadIdx.x & 31;
    const int d = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (d >= ndir) return;
    const double *a = A + (long long)blockIdx.y * Nb;
    const double *row = Bq + (long long)d * Nb;
    double phi = 0.0, sig = 0.0;
    for (int k = lane; k < Nb; k += 32) {
        double v = row[k] * a[k];
        phi += v;
        sig += degree_of(k) * v;
    }
    phi = warp_sum(phi);
    sig = warp_sum(sig);
    if (lane == 0) {
        double w = dirs[d].w;
        img[(long long)blockIdx.y * ndir + d] = make_double2(w * sig / (Rs * 4.0 * kPi), w * phi / (4.0 * kPi));
    }
}

// A block of kSurfThreads = kSurfSplit x kSurfGroup threads covers kSurfTB
// particles (kSurfT per thread); the kSurfSplit thread groups take every
// kSurfSplit-th direction of each staged tile (more warps per SM for the
// same work), and their partial sums are added in group order at the end.
constexpr int kSurfThreads = 256;
constexpr int kSurfSplit = 8;
constexpr int kSurfGroup = kSurfThreads / kSurfSplit;
constexpr int kSurfT = 2;
constexpr int kSurfTB = kSurfGroup * kSurfT;
constexpr int kSurfTile = 256;

__device__ __forceinline__ int find_sys_surf(const SysDesc *sys, int nsys, int item)
{
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (sys[mid].surf_off <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// FP32 form.  For direction u with d = r - Rs u, h = dr/2, a = u.d:
//   sigma image:  Q/|d|, field Q d/|d|^3
//   dipole pair:  (p/dr)(1/A - 1/B) with A = |d + h u|, B = |d - h u|
//                 = -2 p a / (A B (A + B))                  (no cancellation)
//   its field:    (p/dr)((d + h u)/A^3 - (d - h u)/B^3)
//                 = p [ -2 a (A^2 + A B + B^2) / ((A + B) A^3 B^3) d
//                       + (u/2)(1/A^3 + 1/B^3) ]
//
// Each thread takes two directions of its group per step with packed FP32
// instructions (fma/add/mul.rn.f32x2 on the pair); the group's directions
// of a staged tile are stored pair-interleaved: sx = (u_x, u_x', u_y, u_y'),
// sy = (u_z, u_z', Q, Q'), sz = (-2 p, -2 p', p/2, p'/2).  Slots beyond the
// tile hold a direction with Q = p = 0, which contributes exactly zero.
constexpr int kSurfPairs = kSurfTile / kSurfSplit / 2;  // direction pairs per group per tile

__global__ void __launch_bounds__(kSurfThreads, 2) surface_pairs_fp32_kernel(
    const SysDesc *sys, int nsys, const float4 *src_hi, const float4 *src_lo, int ndir, const double4_32a *dirs,
    const double2 *img, float Rs, float h, double *phi_out, double *e_out)
{
    __shared__ float4 sx[kSurfSplit][kSurfPairs], sy[kSurfSplit][kSurfPairs], sz[kSurfSplit][kSurfPairs];
    __shared__ float2 red[kSurfSplit - 1][kSurfT][4][kSurfGroup];  // partial sums of groups 1..
    const int s = find_sys_surf(sys, nsys, blockIdx.x);
    const SysDesc sd = sys[s];
    const int blk = blockIdx.x - sd.surf_off;
    const int gl = threadIdx.x % kSurfGroup;  // particle lane
    const int grp = threadIdx.x / kSurfGroup;  // direction group (uniform per warp)
    float2 RX[kSurfT], RY[kSurfT], RZ[kSurfT];  // particle position, both lanes
    long long idx[kSurfT];
#pragma unroll
    for (int t = 0; t < kSurfT; ++t) {
        long long i = sd.sp_lo + (long long)blk * kSurfTB + t * kSurfGroup + gl;
        const bool ok = i < sd.sp_lo + sd.sp_n;
        idx[t] = ok ? i : -1;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
        if (ok) {
            a = src_hi[sd.src_off + i];
            b = src_lo[sd.src_off + i];
        }
        const float rx = a.x + b.x, ry = a.y + b.y, rz = a.z + b.z;
        RX[t] = make_float2(rx, rx);
        RY[t] = make_float2(ry, ry);
        RZ[t] = make_float2(rz, rz);
    }
    const float2 NRS = make_float2(-Rs, -Rs), HH = make_float2(h * h, h * h);
    const float2 H2 = make_float2(2.f * h, 2.f * h), NH2 = make_float2(-2.f * h, -2.f * h);
    float2 phi[kSurfT], e[kSurfT][3];
#pragma unroll
    for (int t = 0; t < kSurfT; ++t) {
        phi[t] = make_float2(0.f, 0.f);
        e[t][0] = e[t][1] = e[t][2] = make_float2(0.f, 0.f);
    }
    const double2 *im = img + (long long)s * ndir;
    float *fx = reinterpret_cast<float *>(&sx[0][0]), *fy = reinterpret_cast<float *>(&sy[0][0]);
    float *fz = reinterpret_cast<float *>(&sz[0][0]);
    for (int d0 = 0; d0 < ndir; d0 += kSurfTile) {
        const int cnt = min(kSurfTile, ndir - d0);
        __syncthreads();
        for (int j = threadIdx.x; j < kSurfTile; j += kSurfThreads) {
            float ux = 1.f, uy = 0.f, uz = 0.f, Q = 0.f, pw = 0.f;
            if (j < cnt) {
                const double4_32a u = dirs[d0 + j];
                const double2 c = im[d0 + j];
                const bool live = u.w > 0.0;
                ux = (float)u.x;
                uy = (float)u.y;
                uz = (float)u.z;
                Q = live ? (float)c.x : 0.f;
                pw = live ? (float)c.y : 0.f;
            }
            const int g = j % kSurfSplit, k = j / kSurfSplit, kp = k >> 1, ln = k & 1;
            const int base = (g * kSurfPairs + kp) * 4;
            fx[base + ln] = ux;
            fx[base + 2 + ln] = uy;
            fy[base + ln] = uz;
            fy[base + 2 + ln] = Q;
            fz[base + ln] = -2.f * pw;
            fz[base + 2 + ln] = 0.5f * pw;
        }
        __syncthreads();
        const int cg = cnt > grp ? (cnt - grp + kSurfSplit - 1) / kSurfSplit : 0;  // this group's directions
        const int npairs = (cg + 1) >> 1;
        float2 pa[kSurfT], ea[kSurfT][3];
#pragma unroll
        for (int t = 0; t < kSurfT; ++t) {
            pa[t] = make_float2(0.f, 0.f);
            ea[t][0] = ea[t][1] = ea[t][2] = make_float2(0.f, 0.f);
        }
#pragma unroll 2
        for (int kp = 0; kp < npairs; ++kp) {
            const float4 X = sx[grp][kp], Y = sy[grp][kp], Z = sz[grp][kp];
            const float2 ux = make_float2(X.x, X.y), uy = make_float2(X.z, X.w);
            const float2 uz = make_float2(Y.x, Y.y), Q = make_float2(Y.z, Y.w);
            const float2 np2 = make_float2(Z.x, Z.y), hp = make_float2(Z.z, Z.w);
#pragma unroll
            for (int t = 0; t < kSurfT; ++t) {
                const float2 dx = __ffma2_rn(NRS, ux, RX[t]);
                const float2 dy = __ffma2_rn(NRS, uy, RY[t]);
                const float2 dz = __ffma2_rn(NRS, uz, RZ[t]);
                const float2 dd = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                const float2 ad = __ffma2_rn(ux, dx, __ffma2_rn(uy, dy, __fmul2_rn(uz, dz)));
                const float2 base = __fadd2_rn(dd, HH);
                const float2 A2 = __ffma2_rn(H2, ad, base);
                const float2 B2 = __ffma2_rn(NH2, ad, base);
                const float2 ri = make_float2(rsqrt_sfu(dd.x), rsqrt_sfu(dd.y));
                const float2 Ai = make_float2(rsqrt_sfu(A2.x), rsqrt_sfu(A2.y));
                const float2 Bi = make_float2(rsqrt_sfu(B2.x), rsqrt_sfu(B2.y));
                const float2 Aa = __fmul2_rn(A2, Ai), Bb = __fmul2_rn(B2, Bi);
                const float2 sab = __fadd2_rn(Aa, Bb);
                const float2 inv = make_float2(__fdividef(1.f, sab.x), __fdividef(1.f, sab.y));
                const float2 qs = __fmul2_rn(Q, ri);
                const float2 m1 = __fmul2_rn(np2, ad);                                   // -2 p a
                const float2 dip = __fmul2_rn(__fmul2_rn(m1, __fmul2_rn(Ai, Bi)), inv);  // dipole potential
                pa[t] = __fadd2_rn(pa[t], __fadd2_rn(qs, dip));
                const float2 ri3 = __fmul2_rn(__fmul2_rn(ri, ri), ri);
                const float2 Ai3 = __fmul2_rn(__fmul2_rn(Ai, Ai), Ai);
                const float2 Bi3 = __fmul2_rn(__fmul2_rn(Bi, Bi), Bi);
                const float2 S = __fadd2_rn(__ffma2_rn(Aa, Bb, A2), B2);  // A^2 + A B + B^2
                const float2 cd = __fadd2_rn(
                    __fmul2_rn(Q, ri3), __fmul2_rn(__fmul2_rn(__fmul2_rn(__fmul2_rn(m1, S), inv), Ai3), Bi3));
                const float2 cu = __fmul2_rn(hp, __fadd2_rn(Ai3, Bi3));
                ea[t][0] = __fadd2_rn(ea[t][0], __ffma2_rn(cd, dx, __fmul2_rn(cu, ux)));
                ea[t][1] = __fadd2_rn(ea[t][1], __ffma2_rn(cd, dy, __fmul2_rn(cu, uy)));
                ea[t][2] = __fadd2_rn(ea[t][2], __ffma2_rn(cd, dz, __fmul2_rn(cu, uz)));
            }
        }
#pragma unroll
        for (int t = 0; t < kSurfT; ++t) {
            phi[t] = df_add(phi[t], pa[t].x + pa[t].y);
            e[t][0] = df_add(e[t][0], ea[t][0].x + ea[t][0].y);
            e[t][1] = df_add(e[t][1], ea[t][1].x + ea[t][1].y);
            e[t][2] = df_add(e[t][2], ea[t][2].x + ea[t][2].y);
        }
    }
    // add the groups' partial sums in group order
    if (grp > 0) {
#pragma unroll
        for (int t = 0; t < kSurfT; ++t) {
            red[grp - 1][t][0][gl] = phi[t];
            red[grp - 1][t][1][gl] = e[t][0];
            red[grp - 1][t][2][gl] = e[t][1];
            red[grp - 1][t][3][gl] = e[t][2];
        }
    }
    __syncthreads();
    if (grp > 0) return;
#pragma unroll
    for (int t = 0; t < kSurfT; ++t) {
#pragma unroll
        for (int g2 = 0; g2 < kSurfSplit - 1; ++g2) {
            phi[t] = df_add_df(phi[t], red[g2][t][0][gl]);
            e[t][0] = df_add_df(e[t][0], red[g2][t][1][gl]);
            e[t][1] = df_add_df(e[t][1], red[g2][t][2][gl]);
            e[t][2] = df_add_df(e[t][2], red[g2][t][3][gl]);
        }
        if (idx[t] < 0) continue;
        long long o = sd.part_off + idx[t];
        phi_out[o] = (double)phi[t].x + (double)phi[t].y;
        e_out[3 * o] = (double)e[t][0].x + (double)e[t][0].y;
        e_out[3 * o + 1] = (double)e[t][1].x + (double)e[t][1].y;
        e_out[3 * o + 2] = (double)e[t][2].x + (double)e[t][2].y;
    }
}

// FP64 form: the three point images of each direction summed literally; one
// particle per thread, kSurfTB per block (the FP32 kernel's block size).
constexpr int kSurf64Threads = kSurfTB;
__global__ void __launch_bounds__(kSurf64Threads) surface_pairs_fp64_kernel(
    const SysDesc *sys, int nsys, const double4_32a *src64, int ndir, const double4_32a *dirs, const double2 *img,
    double Rs, double dr, double *phi_out, double *e_out)
{
    __shared__ double4_32a su[kSurfTile];
    __shared__ double sp[kSurfTile];
    const int s = find_sys_surf(sys, nsys, blockIdx.x);
    const SysDesc sd = sys[s];
    const int blk = blockIdx.x - sd.surf_off;
    constexpr int T = 1;
    double r[T][3];
    long long idx[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        long long i = sd.sp_lo + (long long)blk * kSurfTB + t * kSurf64Threads + threadIdx.x;
        const bool ok = i < sd.sp_lo + sd.sp_n;
        idx[t] = ok ? i : -1;
        double4_32a a = make_double4_32a(0, 0, 0, 0);
        if (ok) a = src64[sd.src_off + i];
        r[t][0] = a.x;
        r[t][1] = a.y;
        r[t][2] = a.z;
    }
    double phi[T], e[T][3];
#pragma unroll
    for (int t = 0; t < T; ++t) phi[t] = e[t][0] = e[t][1] = e[t][2] = 0.0;
    const double2 *im = img + (long long)s * ndir;
    const double Rin = Rs - 0.5 * dr, Rout = Rs + 0.5 * dr;
    for (int d0 = 0; d0 < ndir; d0 += kSurfTile) {
        int cnt = min(kSurfTile, ndir - d0);
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += kSurf64Threads) {
            double4_32a u = dirs[d0 + j];
            double2 c = im[d0 + j];
            su[j] = make_double4_32a(u.x, u.y, u.z, c.x);
            sp[j] = c.y / dr;
        }
        __syncthreads();
        for (int j = 0; j < cnt; ++j) {
            const double4_32a u = su[j];
            const double pd = sp[j];
            const double R3[3] = {Rs, Rin, Rout};
            const double Q3[3] = {u.w, pd, -pd};
#pragma unroll
            for (int t = 0; t < T; ++t) {
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    double dx = r[t][0] - R3[m] * u.x;
                    double dy = r[t][1] - R3[m] * u.y;
                    double dz = r[t][2] - R3[m] * u.z;
                    double ri = rsqrt(dx * dx + dy * dy + dz * dz);
                    double qr = Q3[m] * ri;
                    phi[t] += qr;
                    double qr3 = qr * ri * ri;
                    e[t][0] += qr3 * dx;
                    e[t][1] += qr3 * dy;
                    e[t][2] += qr3 * dz;
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
        if (idx[t] < 0) continue;
        long long o = sd.part_off + idx[t];
        phi_out[o] = phi[t];
        e_out[3 * o] = e[t][0];
        e_out[3 * o + 1] = e[t][1];
        e_out[3 * o + 2] = e[t][2];
    }
}

// Forces, potentials and per-block energy partials of the particles a call
// owns: the sorted range [sp_lo, sp_lo + sp_n) of each system (all of it,
// except for a part of a target-sharded step).  Target i of a system is its
// i-th particle in spatial order; perm maps it back to the caller's index.
// Block b of system s covers particles [sp_lo + b kFinal, sp_lo + (b + 1) kFinal).
// owned_idx == nullptr: outputs at the caller's indices; otherwise (one
// system) output j is particle sp_lo + j and owned_idx[j] its caller index.
constexpr int kFinalThreads = 256;
constexpr int kFinal = 2048;

__global__ void __launch_bounds__(kFinalThreads) finalize_kernel(const SysDesc *sys, const int *perm, const double *q,
                                                                 const double *phi_tgt, const double *e_part,
                                                                 const double *phi_out, const double *e_out,
                                                                 double *forces, double *pot, long long *owned_idx,
                                                                 double *upart, int nb_max, int *status)
{
    __shared__ double red[32];
    const int s = blockIdx.y;
    const SysDesc sd = sys[s];
    const long long i0 = sd.sp_lo + (long long)blockIdx.x * kFinal;
    const long long i1 = sd.sp_lo + sd.sp_n;
    double u = 0.0;
    bool bad = false;
    for (long long i = i0 + threadIdx.x; i < i1 && i < i0 + kFinal; i += blockDim.x) {
        long long t = sd.tgt_off + i, so = sd.part_off + i;
        const long long ci = sd.part_off + perm[so];  // caller's index
        double qi = q[ci];
        long long o = ci;
        if (owned_idx) {
            o = i - sd.sp_lo;
            owned_idx[o] = perm[so];
        }
        double ph = phi_tgt[t] + phi_out[so];
        double ex = e_part[3 * t] + e_out[3 * so];
        double ey = e_part[3 * t + 1] + e_out[3 * so + 1];
        double ez = e_part[3 * t + 2] + e_out[3 * so + 2];
        if (!isfinite(ph) || !isfinite(ex) || !isfinite(ey) || !isfinite(ez)) bad = true;
        if (forces) {
            forces[3 * o] = qi * ex;
            forces[3 * o + 1] = qi * ey;
            forces[3 * o + 2] = qi * ez;
        }
        if (pot) pot[o] = ph;
        u += qi * ph;
    }
    if (bad) atomicOr(&status[s], ST_COINCIDENT);
    u = block_sum(u, red);
    if (threadIdx.x == 0) upart[(long long)s * nb_max + blockIdx.x] = u;
}

// U = 1/2 sum of the block partials, in block order (of the owned range).
__global__ void energy_kernel(const SysDesc *sys, const double *upart, int nb_max, double *energy, int *status)
{
    const int s = blockIdx.x;
    if (threadIdx.x != 0) return;
    const SysDesc sd = sys[s];
    const int nb = (int)((sd.sp_n + kFinal - 1) / kFinal);
    double u = 0.0;
    for (int b = 0; b < nb; ++b) u += upart[(long long)s * nb_max + b];
    energy[s] = 0.5 * u;
    if (!isfinite(u)) atomicOr(&status[s], ST_COINCIDENT);
}

}  // namespace

int launch_fit_fp64(const SysDesc *sys, int nsys, int bc, int K, int ncols, int Nb, const double *Mp,
                    const double *phi_tgt, const int *mon_inv, double *b_out, double *A, cudaStream_t st)
{
    dim3 grid((ncols + 7) / 8, nsys);
    fit_fp64_kernel<<<grid, 256, 0, st>>>(sys, bc, K, ncols, Nb, Mp, phi_tgt, mon_inv, b_out, A);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

int launch_surface_charges(int nsys, int ndir, int Nb, const double *Bq, const double4_32a *dirs, const double *A,
                           double Rs, double2 *img, cudaStream_t st)
{
    dim3 grid((ndir + 7) / 8, nsys);
    surface_charges_kernel<<<grid, 256, 0, st>>>(ndir, Nb, Bq, dirs, A, Rs, img);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

int surface_targets_per_block() { return kSurfTB; }

int launch_surface_pairs(const SysDesc *sys, int nsys, int total_items, const long long *ns, const float4 *src_hi,
                         const float4 *src_lo, const double4_32a *src64, int ndir, const double4_32a *dirs,
                         const double2 *img, double Rs, double dr, int precision, double *phi_out,
                         double *e_out, cudaStream_t st)
{
    (void)ns;
    if (total_items <= 0) return HSMA_OK;
    if (precision == HSMA_FP64)
        surface_pairs_fp64_kernel<<<total_items, kSurf64Threads, 0, st>>>(sys, nsys, src64, ndir, dirs, img, Rs, dr,
                                                                         phi_out, e_out);
    else
        surface_pairs_fp32_kernel<<<total_items, kSurfThreads, 0, st>>>(
            sys, nsys, src_hi, src_lo, ndir, dirs, img, (float)Rs, (float)(0.5 * dr), phi_out, e_out);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

int finalize_blocks(long long max_n) { return (int)((max_n + kFinal - 1) / kFinal); }

int launch_finalize(const SysDesc *sys, int nsys, long long max_n, const int *perm, const double *q,
                    const double *phi_tgt, const double *e_part, const double *phi_out, const double *e_out,
                    double *forces, double *pot, long long *owned_idx, double *upart, double *energy, int *status,
                    cudaStream_t st)
{
    const int nb_max = finalize_blocks(max_n);
    finalize_kernel<<<dim3(nb_max, nsys), kFinalThreads, 0, st>>>(sys, perm, q, phi_tgt, e_part, phi_out, e_out,
                                                                  forces, pot, owned_idx, upart, nb_max, status);
    HSMA_LAUNCHED();
    energy_kernel<<<nsys, 32, 0, st>>>(sys, upart, nb_max, energy, status);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

}  // namespace hsma

namespace hsma {

namespace {

// Direct evaluation of the far field at the particles: Phi_out(r) =
// sum_k A_k B_k(r) (Eq. "harmonic") and E_out = -grad Phi_out, in FP64.  The
// basis is the orthonormal real solid harmonics of basis_kernel:
//   B = norm_k * Pi_n^m(z, r2) * Re/Im (x + i y)^m   (coordinates / Rs),
// with Pi from its three-term recurrence; the recurrence is differentiated
// alongside for dPi/dz and dPi/d(r2), so that
//   grad B = norm_k [ Pi grad(C_m|S_m) + (C_m|S_m)(dPi/dz e_z + 2 dPi/d(r2) r) ],
//   d/dx (C_m + i S_m) = m (C_{m-1} + i S_{m-1}),
//   d/dy (C_m + i S_m) = i m (C_{m-1} + i S_{m-1}).
__global__ void series_field_kernel(const SysDesc *sys, int nsys, int P, double inv_rs, const double *norm,
                                    const double *A, const float4 *src_hi, const float4 *src_lo,
                                    const double4_32a *src64, double *phi_out, double *e_out)
{
    const int s = blockIdx.y;
    const SysDesc sd = sys[s];
    const long long i = sd.sp_lo + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sd.sp_lo + sd.sp_n) return;
    double x, y, z;
    if (src64) {
        double4_32a p = src64[sd.src_off + i];
        x = p.x; y = p.y; z = p.z;
    } else {
        float4 h = src_hi[sd.src_off + i], l = src_lo[sd.src_off + i];
        x = (double)h.x + (double)l.x;
        y = (double)h.y + (double)l.y;
        z = (double)h.z + (double)l.z;
    }
    x *= inv_rs; y *= inv_rs; z *= inv_rs;
    const double r2 = x * x + y * y + z * z;
    const int Nb = (P + 1) * (P + 1);
    const double *a = A + (long long)s * Nb;
    double phi = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    double cm = 1.0, sm = 0.0, cp = 0.0, sp = 0.0;  // (x+iy)^m and (x+iy)^(m-1)
    double pmm = 1.0;
    for (int m = 0; m <= P; ++m) {
        if (m > 0) {
            cp = cm;
            sp = sm;
            double c2 = cm * x - sm * y;
            sm = sm * x + cm * y;
            cm = c2;
            pmm *= (2.0 * m - 1.0);
        }
        // Pi_{n-1}, Pi_{n-2} and their z / r2 derivatives
        double p1 = 0, p2 = 0, z1 = 0, z2 = 0, q1 = 0, q2 = 0;
        for (int n = m; n <= P; ++n) {
            double pn, dz, dq;
            if (n == m) {
                pn = pmm; dz = 0.0; dq = 0.0;
            } else if (n == m + 1) {
                pn = (2.0 * m + 1.0) * z * pmm;
                dz = (2.0 * m + 1.0) * pmm;
                dq = 0.0;
            } else {
                const double inv = 1.0 / (double)(n - m);
                pn = ((2.0 * n - 1.0) * z * p1 - (n + m - 1.0) * r2 * p2) * inv;
                dz = ((2.0 * n - 1.0) * (p1 + z * z1) - (n + m - 1.0) * r2 * z2) * inv;
                dq = ((2.0 * n - 1.0) * z * q1 - (n + m - 1.0) * (p2 + r2 * q2)) * inv;
            }
            p2 = p1; p1 = pn;
            z2 = z1; z1 = dz;
            q2 = q1; q1 = dq;
            // radial part gradient: dPi/dz e_z + 2 dPi/dr2 (x, y, z)
            const double rx = 2.0 * dq * x, ry = 2.0 * dq * y, rz = dz + 2.0 * dq * z;
            const int kc = n * n + n + m;
            const double ac = a[kc] * norm[kc];
            phi += ac * pn * cm;
            gx += ac * (pn * m * cp + cm * rx);
            gy += ac * (-pn * m * sp + cm * ry);
            gz += ac * (cm * rz);
            if (m > 0) {
                const int ks = n * n + n - m;
                const double as = a[ks] * norm[ks];
                phi += as * pn * sm;
                gx += as * (pn * m * sp + sm * rx);
                gy += as * (pn * m * cp + sm * ry);
                gz += as * (sm * rz);
            }
        }
    }
    const long long o = sd.part_off + i;
    phi_out[o] = phi;
    // gradient w.r.t. the scaled coordinates -> physical: times 1/Rs; E = -grad
    e_out[3 * o] = -gx * inv_rs;
    e_out[3 * o + 1] = -gy * inv_rs;
    e_out[3 * o + 2] = -gz * inv_rs;
}

}  // namespace

// FP32 form of series_field_kernel for the reduced precisions: the fully
// normalised recurrence (the coefficients of basis_df_tables, high words;
// every intermediate stays of order (r/Rs)^n, so no order leaves the FP32
// range) and its derivatives in z and r2,
//   d/dz  Pbar_n = a (Pbar_{n-1} + z d/dz Pbar_{n-1}) - b r2 d/dz Pbar_{n-2},
//   d/dr2 Pbar_n = a z d/dr2 Pbar_{n-1} - b (Pbar_{n-2} + r2 d/dr2 Pbar_{n-2}),
// in FP32 (positions from the split words, coefficients staged in shared
// memory), the sums over n folded into double-float accumulators after every
// m.  FP64 issue is slow on this part; this evaluates the fitted series at
// O(N N_b) FP32 cost.
__global__ void series_field_fp32_kernel(const __grid_constant__ BasisDfTables tabs, const SysDesc *sys, int nsys,
                                         int P, double inv_rs, const double *A, const float4 *src_hi,
                                         const float4 *src_lo, double *phi_out, double *e_out)
{
    extern __shared__ float ssm[];  // [Nb] coefficients A_k, a[m][n], b[m][n] ((P+1)^2 each), D, E
    const int s = blockIdx.y;
    const SysDesc sd = sys[s];
    const int W = P + 1, Nb = W * W;
    float *an = ssm, *ta = ssm + Nb, *tb = ta + W * W, *td = tb + W * W, *te = td + W;
    const double *a = A + (long long)s * Nb;
    for (int k = threadIdx.x; k < Nb; k += blockDim.x) {
        an[k] = (float)a[k];
        ta[k] = tabs.a[k / W][k % W].x;
        tb[k] = tabs.b[k / W][k % W].x;
    }
    for (int k = threadIdx.x; k <= P; k += blockDim.x) {
        td[k] = tabs.d[k].x;
        te[k] = tabs.e[k].x;
    }
    __syncthreads();
    const long long i = sd.sp_lo + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= sd.sp_lo + sd.sp_n) return;
    const float4 h = src_hi[sd.src_off + i], l = src_lo[sd.src_off + i];
    const float ir = (float)inv_rs;
    const float x = (h.x + l.x) * ir, y = (h.y + l.y) * ir, z = (h.z + l.z) * ir;
    const float r2 = fmaf(x, x, fmaf(y, y, z * z));
    float2 phi = make_float2(0.f, 0.f), gx = phi, gy = phi, gz = phi;
    float cm = 1.f, sm = 0.f, cp = 0.f, sp = 0.f;  // (x+iy)^m and (x+iy)^(m-1)
    for (int m = 0; m <= P; ++m) {
        if (m > 0) {
            cp = cm;
            sp = sm;
            const float c2 = cm * x - sm * y;
            sm = sm * x + cm * y;
            cm = c2;
        }
        const float fm = (float)m;
        float p1 = 0.f, p2 = 0.f, z1 = 0.f, z2 = 0.f, q1 = 0.f, q2 = 0.f;
        float fp = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
        const float *am = ta + m * W, *bm = tb + m * W;
        for (int n = m; n <= P; ++n) {
            float pn, dz, dq;
            if (n == m) {
                pn = td[m];
                dz = 0.f;
                dq = 0.f;
            } else if (n == m + 1) {
                pn = te[m] * z;
                dz = te[m];
                dq = 0.f;
            } else {
                const float ca = am[n], cb = bm[n];
                pn = ca * z * p1 - cb * r2 * p2;
                dz = ca * (p1 + z * z1) - cb * r2 * z2;
                dq = ca * z * q1 - cb * (p2 + r2 * q2);
            }
            p2 = p1; p1 = pn;
            z2 = z1; z1 = dz;
            q2 = q1; q1 = dq;
            const float rx = 2.f * dq * x, ry = 2.f * dq * y, rz = dz + 2.f * dq * z;
            const float ac = an[n * n + n + m];
            fp += ac * pn * cm;
            fx += ac * (pn * fm * cp + cm * rx);
            fy += ac * (-pn * fm * sp + cm * ry);
            fz += ac * (cm * rz);
            if (m > 0) {
                const float as = an[n * n + n - m];
                fp += as * pn * sm;
                fx += as * (pn * fm * sp + sm * rx);
                fy += as * (pn * fm * cp + sm * ry);
                fz += as * (sm * rz);
            }
        }
        phi = df_add(phi, fp);
        gx = df_add(gx, fx);
        gy = df_add(gy, fy);
        gz = df_add(gz, fz);
    }
    const long long o = sd.part_off + i;
    phi_out[o] = (double)phi.x + (double)phi.y;
    e_out[3 * o] = -((double)gx.x + (double)gx.y) * inv_rs;
    e_out[3 * o + 1] = -((double)gy.x + (double)gy.y) * inv_rs;
    e_out[3 * o + 2] = -((double)gz.x + (double)gz.y) * inv_rs;
}

int launch_series_field(const SysDesc *sys, int nsys, long long max_n, int P, double Rs, const double *norm,
                        const double *A, const float4 *src_hi, const float4 *src_lo, const double4_32a *src64,
                        double *phi_out, double *e_out, cudaStream_t st)
{
    dim3 grid((unsigned)((max_n + 127) / 128), nsys);
    if (!src64 && src_hi && P <= kBasisTableMaxP) {
        const size_t smem = sizeof(float) * (3 * (size_t)(P + 1) * (P + 1) + 2 * (size_t)(P + 1));
        series_field_fp32_kernel<<<grid, 128, smem, st>>>(basis_df_tables(), sys, nsys, P, 1.0 / Rs, A, src_hi, src_lo,
                                                          phi_out, e_out);
    } else {
        series_field_kernel<<<grid, 128, 0, st>>>(sys, nsys, P, 1.0 / Rs, norm, A, src_hi, src_lo, src64, phi_out,
                                                  e_out);
    }
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

}  // namespace hsma
