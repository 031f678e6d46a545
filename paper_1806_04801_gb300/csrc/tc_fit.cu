// Least-squares fit A = M+ b on the tensor cores (the dense contraction of the
// fit, Sec. II.A/II.C), for all systems of a batch at once:
//   C (ncols x nsys) = M+ (ncols x K) . B (K x nsys),  B(:, s) = b_s.
// Both operands are split into two BF16 words, x = x_hi + x_lo, and the
// product is taken as lo.hi + hi.lo + hi.hi with FP32 accumulation on the
// 5th-generation tensor cores: tcgen05.mma (kind::f16, BF16 inputs, M = 128,
// N = up to 256 systems) issued by one thread, operands in shared memory,
// the accumulator in tensor memory (TMEM), completion through tcgen05.commit
// on an mbarrier, read back with tcgen05.ld.  One refinement step follows:
// r = b - M A1 on the CUDA cores as a compensated dot product (M held as
// FP32 word pairs, every product's rounding error recovered with an FMA,
// the sum's by TwoSum: the result is as accurate as if computed in twice the
// working precision), then A = A1 + M+ r (split-BF16 on the tensor cores as
// the first product).  The residual stays off the tensor cores: their FP32
// accumulation cannot hold it to the ~1e-8 |b| an ill-conditioned fit needs.
// K is padded to a multiple of 16, ncols to 16, nsys to 8 (zeros).
//
// The whole fit is one cooperative launch, one CTA per SM, in five phases
// separated by grid-wide barriers (all CTAs are resident, every wait is
// bounded): (1) the first product -- each CTA takes (row tile, system tile,
// K split) tiles, builds b for its K slab from the monitoring potentials
// while staging it, and writes an FP32 partial; (2) the partials are added
// in split order; (3) the residual, split into BF16; (4) the second
// product; (5) A = A1 +
// the added partials of the second product.  K is split over CTAs so that
// even one system covers the SMs; every sum runs in a fixed order, so
// results do not depend on scheduling.
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
constexpr int kTcThreads = 256;  // warps 0-3 read TMEM lanes 0-127; all eight stage and sum
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

// Stage rows [row0, row0 + R) x columns [k0, k0 + kTcKC) of a row-major
// BF16 matrix (rows of length ld, a multiple of 8; rows >= nrows and columns
// >= ld read as zero) into the core-matrix layout above.  Every 16-byte
// piece is one row of a core matrix.  Loads bypass L1: some operands are
// written by other CTAs of the same launch.
__device__ __forceinline__ void tc_stage(const __nv_bfloat16 *src, int nrows, int ld, int row0, int k0, int R,
                                         unsigned char *dst)
{
    const int pieces = R * (kTcKC / 8);
    constexpr int kBatch = 8;  // loads in flight per thread before the stores
    for (int q0 = threadIdx.x; q0 < pieces; q0 += kBatch * kTcThreads) {
        uint4 v[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int q = q0 + u * kTcThreads;
            const int r = q / (kTcKC / 8), kb = q % (kTcKC / 8);
            const int row = row0 + r, k = k0 + kb * 8;
            v[u] = make_uint4(0u, 0u, 0u, 0u);
            if (q < pieces && row < nrows && k < ld)
                v[u] = __ldcg(reinterpret_cast<const uint4 *>(src + (long long)row * ld + k));
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int q = q0 + u * kTcThreads;
            if (q >= pieces) break;
            const int r = q / (kTcKC / 8), kb = q % (kTcKC / 8);
            *reinterpret_cast<uint4 *>(dst + ((r >> 3) * 8 + kb) * 128 + (r & 7) * 16) = v[u];
        }
    }
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

// M (K x n_cols, FP64) as FP32 word pairs, M ~ hi + lo to ~2^-48.
__global__ void split_rows_kernel(long long n, const double *M, float2 *Mdf)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double v = M[t];
    const float h = (float)v;
    Mdf[t] = make_float2(h, (float)(v - (double)h));
}

// Compensated dot-product accumulation (Ogita, Rump & Oishi, "Accurate sum
// and dot product", 2005, Dot2) of the terms m * a with m a double-float
// value: s carries the FP32 sum, c the sum of the exact rounding errors of
// every product (FMA) and every addition (TwoSum).
// (Intrinsics keep the compiler from fusing the products into the sums,
// which would break the error-free transformations.)
__device__ __forceinline__ void dot2_add(float &s, float &c, float2 m, float a)
{
    const float p = __fmul_rn(m.x, a);
    float ep = fmaf(m.x, a, -p);  // exact error of the high product
    ep = fmaf(m.y, a, ep);        // plus the low word's product
    const float t = __fadd_rn(s, p);
    const float bb = __fsub_rn(t, s);
    const float es = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));  // exact error of s + p
    s = t;
    c = __fadd_rn(c, __fadd_rn(es, ep));
}

// Two compensated partial sums added (the same TwoSum on the FP32 sums).
__device__ __forceinline__ void dot2_merge(float &s, float &c, float s2, float c2)
{
    const float t = __fadd_rn(s, s2);
    const float bb = __fsub_rn(t, s);
    const float es = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(s2, bb));
    s = t;
    c = __fadd_rn(c, __fadd_rn(es, c2));
}

// shared memory: the A operand (two words of 128 x 64), the B operand (two
// words of up to 256 x 64)
constexpr size_t kTcAWord = (size_t)kTcM * kTcKC * 2, kTcBWord = (size_t)kTcNMax * kTcKC * 2;
constexpr size_t kTcSmem = 2 * kTcAWord + 2 * kTcBWord;  // 96 KB
// the dynamic shared memory of a launch also holds the residual's block of
// A1 (ncols x 32 floats) and a row of M per warp, when they fit (ncols <=
// 1205, p <= 33), else the few-systems form's A1 values (ncols x 8)
inline size_t tc_many_smem_bytes(int ncols)
{
    return (size_t)ncols * (32 * sizeof(float) + (kTcThreads / 32) * sizeof(float2));
}
constexpr size_t kTcSmemCap = 226 * 1024;  // the part's limit per CTA, less the static shared memory
inline size_t tc_smem_bytes(int ncols)
{
    const size_t many = tc_many_smem_bytes(ncols);
    return std::max(kTcSmem, many <= kTcSmemCap ? many : (size_t)ncols * 8 * sizeof(float));
}
constexpr long long kBarrierPolls = 8000000;  // x >= 32 ns: a barrier gives up after > 0.25 s

struct TcFitArgs {
    const SysDesc *sys;
    int nsys, periodic, K, Kp, ncols, np, ns8, Nb;
    int mt, nt, rps, split;
    int many_in_smem;                    // residual_many's operands fit in shared memory
    const __nv_bfloat16 *Ahi, *Alo;      // M+ split, np x Kp
    const float2 *Mdf;                   // M (K x ncols) as FP32 word pairs
    const double *phi_tgt;               // near-field potentials (monitoring targets after each system's particles)
    const int *mon_inv;
    double *b_out;                       // nsys x K
    double *A;                           // nsys x Nb
    __nv_bfloat16 *Bhi, *Blo;            // right-hand sides split, ns8 x Kp
    __nv_bfloat16 *Rhi, *Rlo;            // residual split, ns8 x Kp
    float *A1;                           // first product, ns8 x np (system-major)
    float *P;                            // split x ns8 x np partial products (system-major)
    unsigned *bar;                       // [0] cumulative barrier arrivals (zero at launch)
    int *status;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of the cooperative launch.  Every CTA adds its arrival
// to the cumulative count bar[0] (a release reduction) and polls it until
// all CTAs have arrived at barrier number epoch + 1 (bounded: false on a
// timeout).
__device__ bool grid_barrier(unsigned *bar, unsigned &epoch)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = (epoch + 1) * gridDim.x;
        // release: the CTA's writes (ordered before by __syncthreads) precede
        // the arrival; acquire: other CTAs' writes precede what follows
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        long long polls = 0;
        while (ld_acquire_gpu(bar) < target) {
            if (++polls > kBarrierPolls) {
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        s_ok = ok;
    }
    __syncthreads();
    ++epoch;
    return s_ok != 0;
}

// The right-hand sides b_s (Sec. II.A) of every system from the monitoring
// potentials: FP64 into b_out, split into BF16 words into B (ns8 x Kp, zero
// for padding systems and points).  A thread per value.
__device__ void rhs_phase(const TcFitArgs &a)
{
    const long long n = (long long)a.ns8 * a.Kp;
    const long long step = (long long)gridDim.x * kTcThreads;
    const bool periodic = a.periodic != 0;
    constexpr int kB = 4;  // values per thread per pass, their loads issued together
    for (long long t0 = (long long)blockIdx.x * kTcThreads + threadIdx.x; t0 < n; t0 += kB * step) {
        int ia[kB], ib[kB];
        const double *ph[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const long long t = t0 + u * step;
            const int s = (int)(t / a.Kp), i = (int)(t % a.Kp);
            ph[u] = nullptr;
            ia[u] = ib[u] = 0;
            if (t < n && s < a.nsys && i < a.K) {
                ph[u] = a.phi_tgt + __ldg(&a.sys[s].tgt_off) + __ldg(&a.sys[s].n);
                ia[u] = a.mon_inv ? __ldg(a.mon_inv + i) : i;
                ib[u] = periodic ? (a.mon_inv ? __ldg(a.mon_inv + a.K + i) : a.K + i) : 0;
            }
        }
        double v[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u)
            v[u] = ph[u] ? (periodic ? __ldg(ph[u] + ib[u]) - __ldg(ph[u] + ia[u]) : -__ldg(ph[u] + ia[u])) : 0.0;
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const long long t = t0 + u * step;
            if (t >= n) break;
            if (ph[u]) a.b_out[(t / a.Kp) * a.K + t % a.Kp] = v[u];
            split_bf16(v[u], a.Bhi[t], a.Blo[t]);
        }
    }
}

// Read 16 columns of the TMEM accumulator: warp w gets lanes [32 w, 32 w +
// 32), one row per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t tmem, int warp, int c0, uint32_t (&v)[16])
{
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// One tile of a split-BF16 product: rows [m0, m0 + 128) of M+ x systems
// [n0, n0 + N) over the K rounds of split z, accumulated in TMEM and written
// as an FP32 partial to P[z].  second == false: B = b; true: B = the
// residual.  Returns false if a wait ran out.
__device__ bool tc_tile(const TcFitArgs &a, bool second, int t, uint32_t tmem, uint64_t *mbar, uint32_t &phase,
                        unsigned char *smem)
{
    const int z = t % a.split, rest = t / a.split;
    const int ni = rest % a.nt, mi = rest / a.nt;
    const int m0 = mi * kTcM, n0 = ni * kTcNMax;
    const int kbeg = z * a.rps * kTcKC, kend = min(a.Kp, kbeg + a.rps * kTcKC);
    const int N = min(kTcNMax, (a.ns8 - n0 + 15) / 16 * 16);  // MMA N: multiple of 16
    const uint32_t idesc = umma_idesc_bf16(kTcM, N);
    unsigned char *a_hi = smem, *a_lo = smem + kTcAWord;
    unsigned char *b_hi = smem + 2 * kTcAWord, *b_lo = b_hi + kTcBWord;
    for (int k0 = kbeg; k0 < kend; k0 += kTcKC) {
        tc_stage(a.Ahi, a.np, a.Kp, m0, k0, kTcM, a_hi);
        tc_stage(a.Alo, a.np, a.Kp, m0, k0, kTcM, a_lo);
        tc_stage(second ? a.Rhi : a.Bhi, a.ns8, a.Kp, n0, k0, N, b_hi);
        tc_stage(second ? a.Rlo : a.Blo, a.ns8, a.Kp, n0, k0, N, b_lo);
        fence_proxy_async_smem();  // generic writes -> tensor-core (async proxy) reads
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int steps = min(kTcKC, kend - k0) / 16;
            for (int j = 0; j < steps; ++j) {
                const uint32_t off = (uint32_t)(2 * j) * 128u;
                const uint64_t ah = umma_smem_desc(smem_u32(a_hi) + off), al = umma_smem_desc(smem_u32(a_lo) + off);
                const uint64_t bh = umma_smem_desc(smem_u32(b_hi) + off), bl = umma_smem_desc(smem_u32(b_lo) + off);
                umma_bf16(tmem, al, bh, idesc, (k0 > kbeg || j > 0) ? 1 : 0);
                umma_bf16(tmem, ah, bl, idesc, 1);
                umma_bf16(tmem, ah, bh, idesc, 1);
            }
            umma_commit(mbar);  // arrives once the MMAs above have read shared memory and written TMEM
        }
        // the staged operands are rewritten next round: wait for the MMAs
        const bool done = mbar_wait_bounded(mbar, phase);
        phase ^= 1u;
        __syncthreads();
        if (!done) return false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 4) {
        // warp w reads TMEM lanes [32 w, 32 w + 32) = rows m0 + 32 w + lane
        const int row = m0 + warp * 32 + lane;
        // P[z] is system-major (s x np): lanes (consecutive rows) store together
        float *C = a.P + (long long)z * a.np * a.ns8;
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tmem, warp, c0, v);
            if (row < a.np) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + j;
                    if (col < a.ns8) C[(long long)col * a.np + row] = __uint_as_float(v[j]);
                }
            }
        }
    }
    // every warp's TMEM reads precede the next tile's MMAs
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    return true;
}

// The many-systems form of residual_phase: a CTA per (block of 32 systems,
// share of the monitoring points); lanes are systems and run the c loop as
// two interleaved compensated sums, merged at the end.  SMEM: the block's
// A1 values (ncols x 32 floats) and, per warp, the current row of M sit in
// shared memory (ncols up to 1205); otherwise both are read from global
// memory.
template <bool SMEM>
__device__ void residual_many(const TcFitArgs &a, float *sm)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kTcThreads / 32;
    float *sa = sm;  // ncols x 32
    float2 *rows = reinterpret_cast<float2 *>(sm + a.ncols * 32) + (long long)warp * a.ncols;
    const int groups = (a.ns8 + 31) / 32;
    const int per = max(1, (int)gridDim.x / groups);  // CTAs per block of systems
    const int jobs = groups * per;
    for (int job = blockIdx.x; job < jobs; job += gridDim.x) {
        const int g = job / per, part = job % per;
        const int i0 = (int)((long long)part * a.Kp / per), i1 = (int)((long long)(part + 1) * a.Kp / per);
        const int s0 = g * 32, gsz = min(32, a.ns8 - s0);
        const int s = s0 + lane;
        if (SMEM) {
            __syncthreads();  // the previous job's buffers are no longer read
            for (int e = threadIdx.x; e < a.ncols * 32; e += kTcThreads) {
                const int sl = e / a.ncols, c = e % a.ncols;  // consecutive threads: consecutive c
                sa[c * 32 + sl] = sl < gsz ? __ldcg(a.A1 + (long long)(s0 + sl) * a.np + c) : 0.f;
            }
            __syncthreads();
        }
        const float *a1 = a.A1 + (long long)s * a.np;
        for (int i = i0 + warp; i < i1; i += kWarps) {
            const bool live_i = i < a.K;
            const float2 *row = a.Mdf + (long long)i * a.ncols;
            if (SMEM) {
                if (live_i)
                    for (int c = lane; c < a.ncols; c += 32) rows[c] = __ldg(row + c);
                __syncwarp();
            }
            if (lane < gsz) {
                double r = 0.0;
                if (live_i && s < a.nsys) {
                    float sm0 = 0.f, c0 = 0.f, sm1 = 0.f, c1 = 0.f;
                    int c = 0;
                    for (; c + 1 < a.ncols; c += 2) {
                        if (SMEM) {
                            dot2_add(sm0, c0, rows[c], sa[c * 32 + lane]);
                            dot2_add(sm1, c1, rows[c + 1], sa[(c + 1) * 32 + lane]);
                        } else {
                            dot2_add(sm0, c0, __ldg(row + c), __ldcg(a1 + c));
                            dot2_add(sm1, c1, __ldg(row + c + 1), __ldcg(a1 + c + 1));
                        }
                    }
                    if (c < a.ncols) dot2_add(sm0, c0, SMEM ? rows[c] : __ldg(row + c), SMEM ? sa[c * 32 + lane] : __ldcg(a1 + c));
                    dot2_merge(sm0, c0, sm1, c1);
                    r = __ldcg(a.b_out + (long long)s * a.K + i) - ((double)sm0 + (double)c0);
                }
                split_bf16(r, a.Rhi[(long long)s * a.Kp + i], a.Rlo[(long long)s * a.Kp + i]);
            }
            if (SMEM) __syncwarp();  // the row buffer is rewritten for the next point
        }
    }
}

// Residual r_s,i = b_s,i - sum_c M_ic A1_c,s (compensated, dot2_add), split
// into BF16 words at R[s][i]; padding rows and columns are written as zeros.
// The A1 values a CTA needs sit in shared memory (sm, ncols x 32 floats).
//  Few systems (ns8 <= 8): a warp per monitoring point i, lanes over c (the
//    row of M read coalesced), a compensated warp sum per system.
//  Many: residual_many.
__device__ void residual_phase(const TcFitArgs &a, float *sm)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kTcThreads / 32;
    const long long gw = (long long)blockIdx.x * kWarps + warp, nw = (long long)gridDim.x * kWarps;
    if (a.ns8 <= 8) {
        // sm[c * 8 + s] = A1 of system s (< nsys; the others are not read)
        for (int e = threadIdx.x; e < a.ncols * a.nsys; e += kTcThreads) {
            const int sl = e / a.ncols, c = e % a.ncols;
            sm[c * 8 + sl] = __ldcg(a.A1 + (long long)sl * a.np + c);
        }
        __syncthreads();
        for (long long i = gw; i < a.Kp; i += nw) {
            const bool live_i = i < a.K;
            const float2 *row = a.Mdf + i * a.ncols;
            float2 mrow[8];  // this lane's entries c = lane + 32 k of the row
            double bl[8];    // b of system = lane's slot (lanes < nsys), loaded with the row
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c = lane + 32 * k;
                mrow[k] = (live_i && c < a.ncols) ? __ldg(row + c) : make_float2(0.f, 0.f);
                bl[k] = (live_i && k < a.nsys) ? __ldcg(a.b_out + (long long)k * a.K + i) : 0.0;
            }
            for (int s = 0; s < a.ns8; ++s) {
                double r = 0.0;
                if (live_i && s < a.nsys) {
                    float sum = 0.f, err = 0.f;
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int c = lane + 32 * k;
                        if (c < a.ncols) dot2_add(sum, err, mrow[k], sm[c * 8 + s]);
                    }
                    for (int c = lane + 256; c < a.ncols; c += 32) dot2_add(sum, err, __ldg(row + c), sm[c * 8 + s]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const float s2 = __shfl_xor_sync(0xffffffffu, sum, o), c2 = __shfl_xor_sync(0xffffffffu, err, o);
                        dot2_merge(sum, err, s2, c2);
                    }
                    double bs = bl[0];
#pragma unroll
                    for (int k = 1; k < 8; ++k) bs = s == k ? bl[k] : bs;
                    r = bs - ((double)sum + (double)err);
                }
                if (lane == 0) split_bf16(r, a.Rhi[(long long)s * a.Kp + i], a.Rlo[(long long)s * a.Kp + i]);
            }
        }
        return;
    }
    if (a.many_in_smem)
        residual_many<true>(a, sm);
    else
        residual_many<false>(a, sm);
}

// Sum over the splits of P[z][i], in split order (FP32); the loads of eight
// splits are issued before their sums.
__device__ __forceinline__ float split_sum(const TcFitArgs &a, long long i)
{
    const long long n = (long long)a.np * a.ns8;
    float c = 0.f;
    for (int z0 = 0; z0 < a.split; z0 += 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = z0 + u < a.split ? __ldcg(a.P + (long long)(z0 + u) * n + i) : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (z0 + u < a.split) c += v[u];
    }
    return c;
}

// The same sum by a whole warp (for few outputs): lane l adds splits l,
// l + 32, ... in order, then the lanes' sums are added in a fixed tree.
__device__ __forceinline__ float split_sum_warp(const TcFitArgs &a, long long i)
{
    const int lane = threadIdx.x & 31;
    const long long n = (long long)a.np * a.ns8;
    float c = 0.f;
    for (int z = lane; z < a.split; z += 32) c += __ldcg(a.P + (long long)z * n + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    return c;
}

// For every output i < count: out(i, sum of the splits of P at index(i)).
// A thread per output when there are many, a warp per output otherwise.
template <class Index, class Out>
__device__ __forceinline__ void for_split_sums(const TcFitArgs &a, long long count, Index index, Out out)
{
    const long long threads = (long long)gridDim.x * kTcThreads;
    if (count * 4 >= threads || a.split < 8) {
        for (long long i = (long long)blockIdx.x * kTcThreads + threadIdx.x; i < count; i += threads)
            out(i, split_sum(a, index(i)));
        return;
    }
    const long long warps = threads / 32;
    for (long long i = ((long long)blockIdx.x * kTcThreads + threadIdx.x) / 32; i < count; i += warps) {
        const float v = split_sum_warp(a, index(i));
        if ((threadIdx.x & 31) == 0) out(i, v);
    }
}

__global__ void __launch_bounds__(kTcThreads, 1) tc_fit_kernel(TcFitArgs a)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int warp = threadIdx.x >> 5;
    constexpr uint32_t kCols = 256;  // N <= 256
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        mbar_fence_init();
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    uint32_t phase = 0, epoch = 0;
    bool ok = true;
    const int tiles = a.mt * a.nt * a.split;
    const long long nc = (long long)a.np * a.ns8;

    // (0) right-hand sides
    rhs_phase(a);
    ok = grid_barrier(a.bar, epoch) && ok;
    // (1) first product M+ b
    for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) ok = tc_tile(a, false, t, tmem, &mbar, phase, tc_smem);
    ok = grid_barrier(a.bar, epoch) && ok;
    // (2) A1 = the partials added over the splits
    if (ok)
        for_split_sums(a, nc, [](long long i) { return i; }, [&](long long i, float v) { a.A1[i] = v; });
    ok = grid_barrier(a.bar, epoch) && ok;
    // (3) residual r = b - M A1, split into BF16
    if (ok) residual_phase(a, reinterpret_cast<float *>(tc_smem));
    ok = grid_barrier(a.bar, epoch) && ok;
    // (4) correction M+ r
    for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) ok = tc_tile(a, true, t, tmem, &mbar, phase, tc_smem);
    ok = grid_barrier(a.bar, epoch) && ok;
    // (5) A = A1 + correction (A_00 = 0 for a periodic fit, whose constant column is dropped)
    if (ok) {
        const int drop = a.periodic ? 1 : 0;
        const int ncols = a.ncols, np = a.np, Nb = a.Nb;
        for_split_sums(
            a, (long long)ncols * a.nsys,
            [=](long long i) { return (i / ncols) * np + i % ncols; },
            [&](long long i, float v) {
                const long long s = i / ncols, c = i % ncols;
                a.A[s * Nb + c + drop] = (double)__ldcg(a.A1 + s * np + c) + (double)v;
                if (drop && c == 0) a.A[s * Nb] = 0.0;
            });
    } else {
        // give MMAs still in flight a bounded chance to finish before TMEM is freed
        mbar_wait_bounded(&mbar, phase ^ 1u, 200000000LL);
        if (threadIdx.x == 0)
            for (int s = 0; s < a.nsys; ++s) atomicOr(&a.status[s], ST_TIMEOUT);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

}  // namespace

size_t tc_operand_bytes(int K, int ncols) { return (size_t)pad16(ncols) * pad16(K) * sizeof(__nv_bfloat16); }

size_t tc_residual_matrix_bytes(int K, int ncols) { return (size_t)K * ncols * sizeof(float2); }

size_t tc_work_bytes(int K, int ncols, int nsys, int sms)
{
    size_t Kp = pad16(K), np = pad16(ncols), ns8 = pad8(nsys);
    const TcSplit t = tc_split(K, ncols, nsys, sms);
    return 4 * ns8 * Kp * sizeof(__nv_bfloat16) + (size_t)t.split * np * ns8 * sizeof(float) +
           np * ns8 * sizeof(float) + 16 + 8 * 256;  // + rounding of each piece
}

int prepare_tc_operands(int K, int ncols, const double *Mp, const double *Mrow, void *Mp_hi, void *Mp_lo, void *Mdf,
                        cudaStream_t st)
{
    const int Kp = pad16(K), np = pad16(ncols);
    const long long nm = (long long)K * ncols;
    split_rows_kernel<<<(unsigned)((nm + 255) / 256), 256, 0, st>>>(nm, Mrow, (float2 *)Mdf);
    HSMA_LAUNCHED();
    // dynamic shared memory of the fit kernel, set once here (outside any graph capture)
    HSMA_CUDA_TRY(cudaFuncSetAttribute(tc_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemCap));
    long long tot = (long long)np * Kp;
    split_matrix_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(K, ncols, Kp, np, Mp, (__nv_bfloat16 *)Mp_hi,
                                                                       (__nv_bfloat16 *)Mp_lo);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

// The fit of all systems: one cooperative launch of one CTA per SM (the
// grid barriers need every CTA resident; the cooperative launch guarantees
// it).  The barrier counters are cleared on the stream first.
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
    TcFitArgs a;
    a.sys = sys;
    a.nsys = nsys;
    a.periodic = bc == HSMA_BC_PERIODIC ? 1 : 0;
    a.K = K;
    a.Kp = Kp;
    a.ncols = ncols;
    a.np = np;
    a.ns8 = ns8;
    a.Nb = Nb;
    a.mt = ts.mt;
    a.nt = ts.nt;
    a.rps = ts.rps;
    a.split = ts.split;
    a.many_in_smem = tc_many_smem_bytes(ncols) <= kTcSmemCap ? 1 : 0;
    a.Ahi = (const __nv_bfloat16 *)Mp_hi;
    a.Alo = (const __nv_bfloat16 *)Mp_lo;
    a.Mdf = (const float2 *)Mdf;
    a.phi_tgt = phi_tgt;
    a.mon_inv = mon_inv;
    a.b_out = b_out;
    a.A = A;
    a.Bhi = (__nv_bfloat16 *)take((size_t)ns8 * Kp * 2);
    a.Blo = (__nv_bfloat16 *)take((size_t)ns8 * Kp * 2);
    a.Rhi = (__nv_bfloat16 *)take((size_t)ns8 * Kp * 2);
    a.Rlo = (__nv_bfloat16 *)take((size_t)ns8 * Kp * 2);
    a.P = (float *)take((size_t)ts.split * np * ns8 * 4);
    a.A1 = (float *)take((size_t)np * ns8 * 4);
    a.bar = (unsigned *)take(16);
    a.status = status;
    HSMA_CUDA_TRY(cudaMemsetAsync(a.bar, 0, sizeof(unsigned), st));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)sms);
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = tc_smem_bytes(ncols);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    HSMA_CUDA_TRY(cudaLaunchKernelEx(&cfg, tc_fit_kernel, a));
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

}  // namespace hsma
