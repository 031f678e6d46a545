// Least-squares fit A = M+ b on the tensor cores (the dense contraction of the
// fit, Sec. II.A/II.C), for all systems of a batch at once:
//   C (ncols x nsys) = M+ (ncols x K) . B (K x nsys),  B(:, s) = b_s.
// Both operands are split into two BF16 words, x = x_hi + x_lo, and the
// product is taken as hi.hi + hi.lo + lo.hi with FP32 accumulation
// (mma.sync m16n8k16, BF16 inputs, FP32 accumulators).  One refinement step
// follows: r = b - M A in FP64, A += M+ r (again split-BF16 on the tensor
// cores).  K is padded to a multiple of 16, ncols to 16, nsys to 8 (zeros).
#include <cuda_bf16.h>

#include "common.cuh"

namespace hsma {

namespace {

inline int pad16(int v) { return (v + 15) / 16 * 16; }
inline int pad8(int v) { return (v + 7) / 8 * 8; }

__device__ __forceinline__ void split_bf16(double v, __nv_bfloat16 &hi, __nv_bfloat16 &lo)
{
    float f = (float)v;
    hi = __float2bfloat16_rn(f);
    lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
}

__global__ void split_matrix_kernel(int K, int ncols, int Kp, int np, const double *Mp, __nv_bfloat16 *hi,
                                    __nv_bfloat16 *lo)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)np * Kp) return;
    int r = (int)(t / Kp), c = (int)(t % Kp);
    double v = (r < ncols && c < K) ? Mp[(long long)r * K + c] : 0.0;
    split_bf16(v, hi[t], lo[t]);
}

// b_s from the monitoring potentials, stored FP64 and split into BF16 columns.
__global__ void rhs_kernel(const SysDesc *sys, int nsys, int bc, int K, int Kp, const double *phi_tgt,
                           const int *inv, double *b_out, __nv_bfloat16 *bhi, __nv_bfloat16 *blo)
{
    int s = blockIdx.y;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Kp) return;
    double b = 0.0;
    if (s < nsys && i < K) {
        const SysDesc sd = sys[s];
        const double *ph = phi_tgt + sd.tgt_off + sd.n;
        const int a = inv ? inv[i] : i;
        if (bc == HSMA_BC_PERIODIC)
            b = ph[inv ? inv[K + i] : K + i] - ph[a];
        else
            b = -ph[a];
        b_out[(long long)s * K + i] = b;
    }
    split_bf16(b, bhi[(long long)s * Kp + i], blo[(long long)s * Kp + i]);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b)
{
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One warp per 16 x 8 output tile.  A: np x Kp row-major, B: ns8 columns of Kp.
__global__ void tc_gemm_kernel(int Kp, int np, int ns8, const __nv_bfloat16 *Ahi, const __nv_bfloat16 *Alo,
                               const __nv_bfloat16 *Bhi, const __nv_bfloat16 *Blo, float *C /* np x ns8 */)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int tiles_n = ns8 / 8;
    const int tm = warp / tiles_n, tn = warp % tiles_n;
    if (tm * 16 >= np) return;
    const int g = lane >> 2, tg = lane & 3;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int r0 = tm * 16 + g, r1 = r0 + 8;
    const int col = tn * 8 + g;
    for (int k0 = 0; k0 < Kp; k0 += 16) {
        const int ka = k0 + 2 * tg, kb = ka + 8;
        uint32_t ah[4], al[4], bh[2], bl[2];
        ah[0] = pack2(Ahi[(long long)r0 * Kp + ka], Ahi[(long long)r0 * Kp + ka + 1]);
        ah[1] = pack2(Ahi[(long long)r1 * Kp + ka], Ahi[(long long)r1 * Kp + ka + 1]);
        ah[2] = pack2(Ahi[(long long)r0 * Kp + kb], Ahi[(long long)r0 * Kp + kb + 1]);
        ah[3] = pack2(Ahi[(long long)r1 * Kp + kb], Ahi[(long long)r1 * Kp + kb + 1]);
        al[0] = pack2(Alo[(long long)r0 * Kp + ka], Alo[(long long)r0 * Kp + ka + 1]);
        al[1] = pack2(Alo[(long long)r1 * Kp + ka], Alo[(long long)r1 * Kp + ka + 1]);
        al[2] = pack2(Alo[(long long)r0 * Kp + kb], Alo[(long long)r0 * Kp + kb + 1]);
        al[3] = pack2(Alo[(long long)r1 * Kp + kb], Alo[(long long)r1 * Kp + kb + 1]);
        bh[0] = pack2(Bhi[(long long)col * Kp + ka], Bhi[(long long)col * Kp + ka + 1]);
        bh[1] = pack2(Bhi[(long long)col * Kp + kb], Bhi[(long long)col * Kp + kb + 1]);
        bl[0] = pack2(Blo[(long long)col * Kp + ka], Blo[(long long)col * Kp + ka + 1]);
        bl[1] = pack2(Blo[(long long)col * Kp + kb], Blo[(long long)col * Kp + kb + 1]);
        mma_bf16(acc, al, bh);
        mma_bf16(acc, ah, bl);
        mma_bf16(acc, ah, bh);
    }
    const int oc = tn * 8 + 2 * tg;
    C[(long long)r0 * ns8 + oc] = acc[0];
    C[(long long)r0 * ns8 + oc + 1] = acc[1];
    C[(long long)r1 * ns8 + oc] = acc[2];
    C[(long long)r1 * ns8 + oc + 1] = acc[3];
}

// A1 = C; residual r = b - M A1 (FP64), split into BF16 columns.
__global__ void residual_kernel(int nsys, int K, int Kp, int ncols, int ns8, const double *Mrow, const double *b,
                                const float *C, double *A1, __nv_bfloat16 *rhi, __nv_bfloat16 *rlo)
{
    int s = blockIdx.y;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Kp) return;
    double r = 0.0;
    if (s < nsys && i < K) {
        double acc = 0.0;
        const double *row = Mrow + (long long)i * ncols;
        for (int c = 0; c < ncols; ++c) acc += row[c] * (double)C[(long long)c * ns8 + s];
        r = b[(long long)s * K + i] - acc;
        if (i < ncols) A1[(long long)s * ncols + i] = (double)C[(long long)i * ns8 + s];
    }
    split_bf16(r, rhi[(long long)s * Kp + i], rlo[(long long)s * Kp + i]);
}

__global__ void combine_kernel(int nsys, int ncols, int ns8, int Nb, int drop, const double *A1, const float *C2,
                               double *A)
{
    int s = blockIdx.y;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys || c >= ncols) return;
    A[(long long)s * Nb + c + drop] = A1[(long long)s * ncols + c] + (double)C2[(long long)c * ns8 + s];
    if (drop && c == 0) A[(long long)s * Nb] = 0.0;
}

}  // namespace

size_t tc_operand_bytes(int K, int ncols) { return (size_t)pad16(ncols) * pad16(K) * sizeof(__nv_bfloat16); }

size_t tc_work_bytes(int K, int ncols, int nsys)
{
    size_t Kp = pad16(K), np = pad16(ncols), ns8 = pad8(nsys);
    return 2 * ns8 * Kp * sizeof(__nv_bfloat16) * 2 + 2 * np * ns8 * sizeof(float) + (size_t)ncols * nsys * 8 + 4096;
}

int prepare_tc_operands(int K, int ncols, const double *Mp, void *Mp_hi, void *Mp_lo, cudaStream_t st)
{
    int Kp = pad16(K), np = pad16(ncols);
    long long tot = (long long)np * Kp;
    split_matrix_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(K, ncols, Kp, np, Mp, (__nv_bfloat16 *)Mp_hi,
                                                                       (__nv_bfloat16 *)Mp_lo);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

int launch_fit_tc(const SysDesc *sys, int nsys, int bc, int K, int ncols, int Nb, const void *Mp_hi,
                  const void *Mp_lo, const double *Mrow, const double *phi_tgt, const int *mon_inv, double *b_out,
                  double *A, float *work, cudaStream_t st)
{
    const int Kp = pad16(K), np = pad16(ncols), ns8 = pad8(nsys);
    char *w = (char *)work;
    auto take = [&](size_t bytes) {
        char *p = w;
        w += (bytes + 255) / 256 * 256;
        return p;
    };
    __nv_bfloat16 *bhi = (__nv_bfloat16 *)take((size_t)ns8 * Kp * 2);
    __nv_bfloat16 *blo = (__nv_bfloat16 *)take((size_t)ns8 * Kp * 2);
    __nv_bfloat16 *rhi = (__nv_bfloat16 *)take((size_t)ns8 * Kp * 2);
    __nv_bfloat16 *rlo = (__nv_bfloat16 *)take((size_t)ns8 * Kp * 2);
    float *C1 = (float *)take((size_t)np * ns8 * 4);
    float *C2 = (float *)take((size_t)np * ns8 * 4);
    double *A1 = (double *)take((size_t)ncols * nsys * 8);
    const __nv_bfloat16 *ahi = (const __nv_bfloat16 *)Mp_hi, *alo = (const __nv_bfloat16 *)Mp_lo;
    dim3 g1((Kp + 255) / 256, ns8);
    rhs_kernel<<<g1, 256, 0, st>>>(sys, nsys, bc, K, Kp, phi_tgt, mon_inv, b_out, bhi, blo);
    HSMA_LAUNCHED();
    const int warps = (np / 16) * (ns8 / 8);
    tc_gemm_kernel<<<(warps + 3) / 4, 128, 0, st>>>(Kp, np, ns8, ahi, alo, bhi, blo, C1);
    HSMA_LAUNCHED();
    residual_kernel<<<g1, 256, 0, st>>>(nsys, K, Kp, ncols, ns8, Mrow, b_out, C1, A1, rhi, rlo);
    HSMA_LAUNCHED();
    tc_gemm_kernel<<<(warps + 3) / 4, 128, 0, st>>>(Kp, np, ns8, ahi, alo, rhi, rlo, C2);
    HSMA_LAUNCHED();
    dim3 g3((ncols + 127) / 128, nsys);
    combine_kernel<<<g3, 128, 0, st>>>(nsys, ncols, ns8, Nb, bc == HSMA_BC_PERIODIC ? 1 : 0, A1, C2, A);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

}  // namespace hsma
