// Least-squares fit A = M+ b on the tensor cores (the dense contraction of the
// fit, Sec. II.A/II.C), for all systems of a batch at once:
//   C (ncols x nsys) = M+ (ncols x K) . B (K x nsys),  B(:, s) = b_s.
// Both operands are split into two BF16 words, x = x_hi + x_lo, and the
// product is taken as lo.hi + hi.lo + hi.hi with FP32 accumulation on the
// 5th-generation tensor cores: tcgen05.mma (kind::f16, BF16 inputs, M = 128,
// N = up to 256 systems) issued by one thread, operands in shared memory,
// the accumulator in tensor memory (TMEM), completion through tcgen05.commit
// on an mbarrier, read back with tcgen05.ld.  One refinement step follows:
// r = b - M A in double-float arithmetic on the FP32 pipe, A += M+ r (again
// split-BF16 on the tensor cores).
// K is padded to a multiple of 16, ncols to 16, nsys to 8 (zeros).
#include <cuda_bf16.h>

#include <algorithm>

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

// ---------------------------------------------------------------- tcgen05
// Shared-memory operand layout (no swizzle, K-major): a tile of R rows x 64 K
// elements is stored as core matrices of 8 rows x 8 elements (8 rows of 16
// bytes, 128 contiguous bytes); core matrix (row group g, K block kb) sits at
// byte (g * 8 + kb) * 128.  So the K-direction core-matrix stride (leading
// byte offset) is 128 B and the row-group stride (stride byte offset) is
// 1024 B; one MMA (K = 16) starts at K block 2j.
constexpr int kTcM = 128;          // rows of M+ per CTA (MMA M)
constexpr int kTcKC = 64;          // K elements staged per round
constexpr int kTcNMax = 256;       // systems per CTA (MMA N <= 256)
constexpr int kTcThreads = 128;
constexpr uint32_t kTcLBO = 128, kTcSBO = 1024;

__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);           // start address >> 4, bits [0,14)
    d |= (uint64_t)(kTcLBO >> 4) << 16;                  // leading (K) byte offset >> 4, bits [16,30)
    d |= (uint64_t)(kTcSBO >> 4) << 32;                  // stride (row group) byte offset >> 4, bits [32,46)
    d |= (uint64_t)1 << 46;                              // descriptor version for this architecture
    return d;                                            // base offset 0, layout: no swizzle
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 in bits [17,23), M >> 4 in bits [24,29).
__device__ __forceinline__ uint32_t umma_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Stage rows [row0, row0 + R) x K [k0, k0 + kTcKC) of a row-major BF16
// matrix (rows of length Kp, rows >= nrows and K >= Kp read as zero) into
// the core-matrix layout above.  Every 16-byte piece is one row of a core
// matrix.
__device__ __forceinline__ void tc_stage(const __nv_bfloat16 *src, int nrows, int Kp, int row0, int k0, int R,
                                         unsigned char *dst)
{
    const int pieces = R * (kTcKC / 8);
    for (int q = threadIdx.x; q < pieces; q += kTcThreads) {
        const int r = q / (kTcKC / 8), kb = q % (kTcKC / 8);
        const int row = row0 + r, k = k0 + kb * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (row < nrows && k < Kp) v = *reinterpret_cast<const uint4 *>(src + (long long)row * Kp + k);
        *reinterpret_cast<uint4 *>(dst + ((r >> 3) * 8 + kb) * 128 + (r & 7) * 16) = v;
    }
}

// One CTA: rows [m0, m0 + 128) x systems [n0, n0 + N) of the product over
// the K rounds [z rps, (z + 1) rps) (split K, z = blockIdx.z).  A: np x Kp,
// B: ns8 rows (one per system) of Kp; P: [split][np x ns8] FP32 partials.
__global__ void __launch_bounds__(kTcThreads) tc_gemm_kernel(int Kp, int np, int ns8, const __nv_bfloat16 *Ahi,
                                                             const __nv_bfloat16 *Alo, const __nv_bfloat16 *Bhi,
                                                             const __nv_bfloat16 *Blo, int rps, float *P,
                                                             int *status, int nsys)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int m0 = blockIdx.x * kTcM, n0 = blockIdx.y * kTcNMax;
    const int N = min(kTcNMax, (ns8 - n0 + 15) / 16 * 16);          // MMA N: multiple of 16
    const uint32_t tcols = N <= 32 ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u));
    unsigned char *a_hi = tc_smem, *a_lo = a_hi + kTcM * kTcKC * 2;
    unsigned char *b_hi = a_lo + kTcM * kTcKC * 2, *b_lo = b_hi + kTcNMax * kTcKC * 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = umma_idesc_bf16(kTcM, N);
    uint32_t phase = 0;
    bool ok = true;
    const int kbeg = blockIdx.z * rps * kTcKC, kend = min(Kp, kbeg + rps * kTcKC);
    float *C = P + (long long)blockIdx.z * np * ns8;
    for (int k0 = kbeg; k0 < kend; k0 += kTcKC) {
        tc_stage(Ahi, np, Kp, m0, k0, kTcM, a_hi);
        tc_stage(Alo, np, Kp, m0, k0, kTcM, a_lo);
        tc_stage(Bhi, ns8, Kp, n0, k0, N, b_hi);
        tc_stage(Blo, ns8, Kp, n0, k0, N, b_lo);
        fence_proxy_async_smem();  // generic writes -> tensor-core (async proxy) reads
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int steps = min(kTcKC, Kp - k0) / 16;
            for (int j = 0; j < steps; ++j) {
                const uint32_t off = (uint32_t)(2 * j) * 128u;
                const uint64_t ah = umma_smem_desc(smem_u32(a_hi) + off), al = umma_smem_desc(smem_u32(a_lo) + off);
                const uint64_t bh = umma_smem_desc(smem_u32(b_hi) + off), bl = umma_smem_desc(smem_u32(b_lo) + off);
                umma_bf16(tmem, al, bh, idesc, (k0 > kbeg || j > 0) ? 1 : 0);
                umma_bf16(tmem, ah, bl, idesc, 1);
                umma_bf16(tmem, ah, bh, idesc, 1);
            }
            umma_commit(&bar);  // arrives once the MMAs above have read shared memory and written TMEM
        }
        // the staged operands are rewritten next round: wait for the MMAs
        if (!mbar_wait_bounded(&bar, phase)) ok = false;
        phase ^= 1u;
        __syncthreads();
        if (!ok) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // warp w reads TMEM lanes [32 w, 32 w + 32) = rows m0 + 32 w + lane
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < np) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + j;
                    if (col < ns8) C[(long long)row * ns8 + col] = __uint_as_float(v[j]);
                }
            }
        }
    } else {
        // give MMAs still in flight a bounded chance to finish before TMEM is freed
        mbar_wait_bounded(&bar, phase ^ 1u, 200000000LL);
        if (threadIdx.x == 0)
            for (int s2 = n0; s2 < min(nsys, n0 + N); ++s2) atomicOr(&status[s2], ST_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

constexpr size_t kTcSmem = (size_t)2 * kTcM * kTcKC * 2 + (size_t)2 * kTcNMax * kTcKC * 2;

// C = sum of the split-K partials, in split order (deterministic).
__global__ void tc_reduce_kernel(long long n, int split, const float *P, float *C)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float c = 0.f;
    for (int z = 0; z < split; ++z) c += P[(long long)z * n + i];
    C[i] = c;
}

// Split of the K rounds over CTAs: enough CTAs to cover the SMs once, every
// CTA at least one round.
struct TcSplit {
    int mt, nt, rounds, rps, split;
};
TcSplit tc_split(int K, int ncols, int nsys, int sms)
{
    TcSplit t;
    const int Kp = pad16(K), np = pad16(ncols), ns8 = pad8(nsys);
    t.mt = (np + kTcM - 1) / kTcM;
    t.nt = (ns8 + kTcNMax - 1) / kTcNMax;
    t.rounds = (Kp + kTcKC - 1) / kTcKC;
    int want = std::max(1, std::min(t.rounds, (sms + t.mt * t.nt - 1) / (t.mt * t.nt)));
    t.rps = (t.rounds + want - 1) / want;
    t.split = (t.rounds + t.rps - 1) / t.rps;
    return t;
}

// A1 = C; residual r = b - M A1 in double-float arithmetic on the FP32 pipe
// (M held as FP32 word pairs, each product split exactly with an FMA, sums
// by TwoSum; ~1e-14 relative, like FP64 at a fraction of its cost on this
// part), split into BF16 columns.
__device__ __forceinline__ float2 df_mul_f(float2 m, float c)
{
    const float p = m.x * c;
    float e = fmaf(m.x, c, -p);  // exact error of the high product
    e = fmaf(m.y, c, e);
    const float h = p + e;
    return make_float2(h, e - (h - p));
}

__global__ void residual_kernel(int nsys, int K, int Kp, int ncols, int ns8, const float2 *Mdf, const double *b,
                                const float *C, double *A1, __nv_bfloat16 *rhi, __nv_bfloat16 *rlo)
{
    int s = blockIdx.y;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Kp) return;
    double r = 0.0;
    if (s < nsys && i < K) {
        float2 acc = make_float2(0.f, 0.f);
        const float2 *row = Mdf + (long long)i * ncols;
        for (int c = 0; c < ncols; ++c) acc = df_add_df(acc, df_mul_f(row[c], C[(long long)c * ns8 + s]));
        const double bi = b[(long long)s * K + i];
        const float bh = (float)bi;
        const float2 bdf = make_float2(bh, (float)(bi - (double)bh));
        const float2 rd = df_add_df(bdf, make_float2(-acc.x, -acc.y));
        r = (double)rd.x + (double)rd.y;
        if (i < ncols) A1[(long long)s * ncols + i] = (double)C[(long long)i * ns8 + s];
    }
    split_bf16(r, rhi[(long long)s * Kp + i], rlo[(long long)s * Kp + i]);
}

// M (K x n_cols, FP64) as FP32 word pairs.
__global__ void split_rows_kernel(long long n, const double *M, float2 *Mdf)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double v = M[t];
    const float h = (float)v;
    Mdf[t] = make_float2(h, (float)(v - (double)h));
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

size_t tc_residual_matrix_bytes(int K, int ncols) { return (size_t)K * ncols * sizeof(float2); }

size_t tc_work_bytes(int K, int ncols, int nsys, int sms)
{
    size_t Kp = pad16(K), np = pad16(ncols), ns8 = pad8(nsys);
    const TcSplit t = tc_split(K, ncols, nsys, sms);
    return 2 * ns8 * Kp * sizeof(__nv_bfloat16) * 2 + 2 * np * ns8 * sizeof(float) + (size_t)ncols * nsys * 8 +
           (size_t)t.split * np * ns8 * sizeof(float) + 16 * 256;  // + rounding of each piece
}

int prepare_tc_operands(int K, int ncols, const double *Mp, const double *Mrow, void *Mp_hi, void *Mp_lo, void *Mdf,
                        cudaStream_t st)
{
    const long long nm = (long long)K * ncols;
    split_rows_kernel<<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(nm, Mrow, (float2 *)Mdf);
    HSMA_LAUNCHED();
    // dynamic shared memory of the GEMM, set once here (outside any graph capture)
    HSMA_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
    int Kp = pad16(K), np = pad16(ncols);
    long long tot = (long long)np * Kp;
    split_matrix_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(K, ncols, Kp, np, Mp, (__nv_bfloat16 *)Mp_hi,
                                                                       (__nv_bfloat16 *)Mp_lo);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

int launch_fit_tc(const SysDesc *sys, int nsys, int bc, int K, int ncols, int Nb, const void *Mp_hi,
                  const void *Mp_lo, const void *Mdf, const double *phi_tgt, const int *mon_inv, double *b_out,
                  double *A, float *work, int *status, int sms, cudaStream_t st)
{
    const TcSplit ts = tc_split(K, ncols, nsys, sms);
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
    float *Pz = (float *)take((size_t)ts.split * np * ns8 * 4);
    const __nv_bfloat16 *ahi = (const __nv_bfloat16 *)Mp_hi, *alo = (const __nv_bfloat16 *)Mp_lo;
    dim3 g1((Kp + 255) / 256, ns8);
    rhs_kernel<<<g1, 256, 0, st>>>(sys, nsys, bc, K, Kp, phi_tgt, mon_inv, b_out, bhi, blo);
    HSMA_LAUNCHED();
    const dim3 gg(ts.mt, ts.nt, ts.split);
    const long long nc = (long long)np * ns8;
    const unsigned gr = (unsigned)((nc + 255) / 256);
    tc_gemm_kernel<<<gg, kTcThreads, kTcSmem, st>>>(Kp, np, ns8, ahi, alo, bhi, blo, ts.rps, Pz, status, nsys);
    HSMA_LAUNCHED();
    tc_reduce_kernel<<<gr, 256, 0, st>>>(nc, ts.split, Pz, C1);
    HSMA_LAUNCHED();
    residual_kernel<<<g1, 256, 0, st>>>(nsys, K, Kp, ncols, ns8, (const float2 *)Mdf, b_out, C1, A1, rhi, rlo);
    HSMA_LAUNCHED();
    tc_gemm_kernel<<<gg, kTcThreads, kTcSmem, st>>>(Kp, np, ns8, ahi, alo, rhi, rlo, ts.rps, Pz, status, nsys);
    HSMA_LAUNCHED();
    tc_reduce_kernel<<<gr, 256, 0, st>>>(nc, ts.split, Pz, C2);
    HSMA_LAUNCHED();
    dim3 g3((ncols + 127) / 128, nsys);
    combine_kernel<<<g3, 128, 0, st>>>(nsys, ncols, ns8, Nb, bc == HSMA_BC_PERIODIC ? 1 : 0, A1, C2, A);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

}  // namespace hsma
