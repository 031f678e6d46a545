// Internal declarations shared by the CUDA translation units of libhsma.
// Not part of the public ABI (include/hsma.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/hsma.h"

namespace hsma {

// ----------------------------------------------------------------- launch
extern std::atomic<long long> g_launches;  // kernels issued by this library

#define HSMA_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) {                              \
            hsma::set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
            return (_e == cudaErrorMemoryAllocation) ? HSMA_E_OOM : HSMA_E_CUDA; \
        }                                                     \
    } while (0)

#define HSMA_LAUNCHED() hsma::g_launches.fetch_add(1, std::memory_order_relaxed)

// Every device and pinned-host allocation or free of this library goes
// through these wrappers, which count the calls (hsma_allocation_calls), so
// that a test can show that an entry point allocates nothing.
extern std::atomic<long long> g_alloc_calls;
template <class T>
inline cudaError_t dev_malloc(T **p, size_t bytes)
{
    g_alloc_calls.fetch_add(1, std::memory_order_relaxed);
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}
inline cudaError_t dev_free(void *p)
{
    g_alloc_calls.fetch_add(1, std::memory_order_relaxed);
    return cudaFree(p);
}
template <class T>
inline cudaError_t host_malloc(T **p, size_t bytes)
{
    g_alloc_calls.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocHost(reinterpret_cast<void **>(p), bytes);
}
inline cudaError_t host_free(void *p)
{
    g_alloc_calls.fetch_add(1, std::memory_order_relaxed);
    return cudaFreeHost(p);
}

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// Device status bits, one int per system; the host maps them to codes.
enum : int {
    ST_NONNEUTRAL = 1,
    ST_OUT_OF_BOX = 2,
    ST_COINCIDENT = 4,
    ST_TIMEOUT = 8,
    ST_CAPACITY = 16,
    ST_STALE = 32,  // reused in-set no longer valid (a particle moved >= the skin, or charges changed)
};

// ------------------------------------------------------------ batch layout
// One record per system of a batch (a single-system call is a batch of one).
struct SysDesc {
    long long n;            // particles
    long long part_off;     // first particle in the concatenated inputs/outputs
    long long src_off;      // first in-set slot (capacity n * n_shifts)
    long long tgt_off;      // first target slot: n particles then n_mon monitors
    long long partial_off;  // first partial record: nchunks * (n + n_mon)
    long long cnt_off;      // first in-set block count: n_shifts * nblk
    long long hist_off;     // first radix-sort histogram entry: 256 * nblk
    long long tile_off;     // first tile bounding box: ceil(n * n_shifts / tile)
    long long sp_lo;        // far-field (surface / series) particles: sorted range [sp_lo, sp_lo + sp_n)
    long long sp_n;
    int gbits;              // Morton grid of 2^gbits cells per axis
    int pb_lo;              // first particle target block of this call (target sharding)
    int mb_lo;              // first monitoring target block of this call
    int pad0;
    int nchunks;            // source chunks of the near-field sums
    int ntb;                // target blocks (particles, then monitors)
    int ntb_part;           // target blocks holding particles
    int nblk;               // in-set blocks per shift
    int item_off;           // first near-field work item of this system
    int surf_off;           // first surface work item of this system
};

// --------------------------------------------------------- numeric helpers
// Error-free transformation a + b = s + e (Knuth's TwoSum), in FP32.  Used to
// fold FP32 partial sums into a double-float (hi, lo) accumulator.
__device__ __forceinline__ float2 df_add(float2 acc, float x)
{
    float s = __fadd_rn(acc.x, x);
    float bb = __fsub_rn(s, acc.x);
    float e = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    return make_float2(s, __fadd_rn(acc.y, e));
}

// Double-float sum of two double-float values (TwoSum of the high words, low
// words added to the error term, renormalised): ~2^-44 relative.
__device__ __forceinline__ float2 df_add_df(float2 a, float2 b)
{
    const float s = __fadd_rn(a.x, b.x);
    const float bb = __fsub_rn(s, a.x);
    float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    const float h = __fadd_rn(s, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}

// Right-hand side of the least-squares fit at monitoring point i (Sec. II.A):
// periodic b_i = Phi_in(x~_i) - Phi_in(x_i) (the periodicity residual),
// grounded b_i = -Phi_in(x_i).  ph: the monitoring-target potentials of one
// system (the K points, then their K partners), in the pair kernel's target
// order; inv maps a point's index to its slot there (nullptr: identity).
__device__ __forceinline__ double rhs_at(const double *ph, const int *inv, int K, int i, bool periodic)
{
    const int a = inv ? inv[i] : i;
    if (!periodic) return -ph[a];
    const int b = inv ? inv[K + i] : K + i;
    return ph[b] - ph[a];
}

// Reciprocal square root on the special-function unit.
__device__ __forceinline__ float rsqrt_sfu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Split an FP64 value into two FP32 words whose sum represents it to ~2^-48.
__device__ __forceinline__ void split_f64(double v, float &hi, float &lo)
{
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
}

// ------------------------------------------------- mbarrier / bulk copies
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared, completing on the mbarrier.  Both addresses
// must be 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after ~max_cycles SM clocks
// (and after a fixed number of polls), returning false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  long long max_cycles = 4000000000LL)
{
    long long t0 = clock64();
    for (int it = 0; it < (1 << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > max_cycles) return false;
    }
    return false;
}

// Deterministic block-wide sum of doubles (blockDim.x a multiple of 32, <= 1024).
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v, double *scratch /* >= 32 */)
{
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    double r = (threadIdx.x < (unsigned)nw) ? scratch[threadIdx.x] : 0.0;
    if (wid == 0) r = warp_sum(r);
    if (threadIdx.x == 0) scratch[0] = r;
    __syncthreads();
    r = scratch[0];
    __syncthreads();
    return r;
}

// Exclusive prefix sum of h[0, total) in place by one block (blockDim a
// multiple of 32, <= 1024); returns the sum of all entries.  Each thread
// scans kPer consecutive entries per round, so a round covers
// kPer * blockDim entries with two block barriers.
__device__ __forceinline__ long long block_scan_inplace(int *h, long long total, int *wsum /* [32] */,
                                                        long long *carry_s)
{
    constexpr int kPer = 8;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long carry = 0;
    for (long long base = 0; base < total; base += (long long)blockDim.x * kPer) {
        const long long t0 = base + (long long)threadIdx.x * kPer;
        int v[kPer];
        int sum = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            v[k] = (t0 + k < total) ? h[t0 + k] : 0;
            sum += v[k];
        }
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int w = (lane < nw) ? wsum[lane] : 0;
            int wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += u;
            }
            wsum[lane] = wi - w;  // exclusive prefix of the warp sums
            if (lane == 31) *carry_s = carry + wi;
        }
        __syncthreads();
        long long e = carry + wsum[wid] + incl - sum;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            if (t0 + k < total) h[t0 + k] = (int)e;
            e += v[k];
        }
        carry = *carry_s;
        __syncthreads();  // wsum and carry_s are rewritten next round
    }
    return carry;
}

// ------------------------------------------------ kernel launch interfaces
// (defined in the .cu files; all enqueue on `st` and return HSMA_OK or a code)

struct Geometry {
    double L[3];
    double Rs;
    int bc;
};

// plan_kernels.cu
int launch_monitor_sphere(int K, double R0, const double L[3], double4_32a *out64, float4 *hi, float4 *lo,
                          cudaStream_t st);
int launch_monitor_faces(const int cnt[6], const double L[3], double4_32a *out64, float4 *hi, float4 *lo,
                         cudaStream_t st);
int launch_quadrature(int F2, int F1, double Rs, double4_32a *dirs, cudaStream_t st);
// Coefficients of the fully normalised recurrence of the orthonormal real
// solid harmonics, Pbar_n^m = norm(n, m) Pi_n^m (every order up to
// kBasisTableMaxP, independent of a plan's P), each as an FP32 pair hi + lo:
//   Pbar_m^m = D_m,  Pbar_{m+1}^m = E_m z,
//   Pbar_n^m = a_nm z Pbar_{n-1}^m - b_nm r2 Pbar_{n-2}^m  (n >= m + 2),
//   a_nm = sqrt((4n^2 - 1)/(n^2 - m^2)),
//   b_nm = sqrt((2n+1)((n-1)^2 - m^2)/((2n-3)(n^2 - m^2))),
//   D_0 = 1/sqrt(4 pi), D_m = D_{m-1} sqrt((2m+1)/(2m)) (times sqrt 2 at m = 1),
//   E_m = sqrt(2m+3) D_m.
// Passed to kernels by value (27.5 KB of parameters).
constexpr int kBasisTableMaxP = 40;
struct BasisDfTables {
    float2 a[kBasisTableMaxP + 1][kBasisTableMaxP + 1];  // a_nm at [m][n] (n >= m + 2)
    float2 b[kBasisTableMaxP + 1][kBasisTableMaxP + 1];  // b_nm at [m][n]
    float2 d[kBasisTableMaxP + 1];                       // D_m
    float2 e[kBasisTableMaxP + 1];                       // E_m
};
const BasisDfTables &basis_df_tables();  // computed once on the host, in FP64

// orthonormalisation constant of the real solid harmonic (n, m), m >= 0:
// sqrt((2 - delta_m0)(2n+1)/(4 pi) (n-m)!/(n+m)!)
double basis_norm(int n, int m);
int launch_basis(int P, double Rs, long long np, const double *pts, int pts_stride, double *out, long long ld,
                 cudaStream_t st);
// the same basis in double-float arithmetic on the FP32 pipe (no norm table)
int launch_basis_df(int P, double Rs, long long np, const double *pts, int pts_stride, double *out, long long ld,
                    cudaStream_t st);
int launch_fitting_matrix(int K, int Nb, int ncols, int drop, const double *Bx, const double *Bxt,
                          double *Mcol, double *Mrow, cudaStream_t st);
int build_pseudo_inverse(int K, int n, double *Wcol, double *Mp, double *cond, int *rank_ok,
                         cudaStream_t st);

// sort.cu
struct SortArgs {
    const SysDesc *sys;
    int nsys;
    const double *xyz;
    Geometry g;
    int *keys, *vals;       // in: unused; out: sorted keys and the permutation
    int *keys2, *vals2;     // ping-pong buffers
    int *hist;
};
int launch_sort_particles(const SortArgs &a, int nblk_max, cudaStream_t st);
int launch_tile_boxes(const SysDesc *sys, int nsys, long long max_tiles, const long long *ns, const float4 *src_hi,
                      int tile, float4 *boxes, cudaStream_t st);
int launch_gather_targets(int n, const int *perm, const double4_32a *in64, const float4 *inhi, const float4 *inlo,
                          double4_32a *out64, float4 *outhi, float4 *outlo, cudaStream_t st);
int launch_array_boxes(int n, const float4 *hi, int block, float4 *boxes, cudaStream_t st);

// inset.cu
struct InsetArgs {
    const SysDesc *sys;
    int nsys;
    int nblk_max;
    const double *xyz;
    const double *q;
    const int *perm;        // sorted position -> particle index within its system
    const int4 *shifts;
    int n_shifts;
    Geometry g;
    int *counts;
    long long *ns;
    float4 *src_hi;
    float4 *src_lo;
    double4_32a *src64;
    int *status;
    double4_32a *cen;       // [n] scratch: centred (x, y, z, q) in spatial order
    float4 *cenf;           // [n] the same rounded to FP32 (the guarded in-sphere test)
    double2 *qsums;         // [blocks] per particle block: (sum q, sum |q|)
    int2 *cand = nullptr;   // candidate pass only: (spatial index, shift) of each hit
};
int launch_inset(const InsetArgs &a, cudaStream_t st);
// The candidate list of a reusable in-set: the same count/scan/scatter over
// a's shifts and radius (the caller passes the enlarged sphere and shift
// table, its own counts / ns buffers and a.cand), after launch_inset of the
// same step has filled cen / cenf.
int launch_inset_candidates(const InsetArgs &a, cudaStream_t st);

// In-set regenerated from a candidate list (single system): image positions
// from the particles' current positions, continued without wrapping from the
// positions of the list's build; the candidates inside Rs, compacted in
// list order (inset.cu).
struct RegenArgs {
    long long n, cap;        // particles; in-set slots of the workspace
    long long cap_cand;      // candidate list capacity
    const long long *ncand;  // device: candidates in the list
    const int2 *cand;        // (spatial index, shift index)
    const int4 *shifts;
    const int *perm;         // spatial index -> caller index (of the build)
    const double4_32a *x0;   // centred positions and charges at the build, spatial order
    const double *xyz, *q;   // current positions (box frame) and charges, caller order
    Geometry g;              // the sphere Rs of the step
    double skin;             // a particle displaced by >= skin makes the list stale
    int *counts;             // [candidate blocks] scratch
    double4_32a *u;          // [n] scratch: continued positions and charges, spatial order
    float4 *src_hi, *src_lo;
    double4_32a *src64;
    long long *ns;
    int *status;
};
int launch_inset_regen(const RegenArgs &r, cudaStream_t st);

// pair.cu
struct PairArgs {
    const SysDesc *sys;
    int nsys;
    int total_items;
    const long long *ns;
    const float4 *src_hi;
    const float4 *src_lo;
    const double4_32a *src64;
    const float4 *ext_hi;   // external targets (monitoring points), shared by all systems
    const float4 *ext_lo;
    const double4_32a *ext64;
    int n_ext;
    int ext_field;          // external targets also need the field
    int ext_skip_zero;      // skip pairs at distance exactly zero for external targets
    const float4 *boxes = nullptr;  // FP32 form: box of every source tile (lo, hi), or null
    const float4 *ext_boxes = nullptr;  // box of every block of external targets, or null
    int stall_test = 0;             // test hook: wait on a barrier nothing arrives at (bounded)
    float far2 = 0.f;               // tiles at least sqrt(far2) from the target block skip the low words
    int one_item = 0;               // 1: CTA b does work item b and exits (grid = total_items), so that
                                    // work on other streams gets SMs between items
    float4 *partials;       // 2 x float4 (FP32) or 1 x double4_32a (FP64) per record
    int *next_item;
    int *status;
};
// variant (FP32 form): one of the codes pair_variant_valid accepts; it fixes
// the targets per thread -- 4 (blocks and tiles of 512), 3 (384) or 2 (256) --
// the inner loop (scalar or packed f32x2) and the CTAs per SM.
int launch_pair(const PairArgs &a, int precision, int variant, int grid, cudaStream_t st);
bool pair_variant_valid(int variant);
int pair_targets_per_block(int precision, int variant = 4);
int pair_max_ctas_per_sm(int precision, int variant = 4);
int launch_partial_reduce(const SysDesc *sys, int nsys, long long max_tgt, int n_ext, const float4 *partials,
                          int precision, double *phi_tgt, double *e_part, cudaStream_t st);

// fit_surface.cu
// mon_inv[i]: slot of monitoring target i among the (spatially ordered)
// external targets the pair kernel used, or null for the identity.
int launch_fit_fp64(const SysDesc *sys, int nsys, int bc, int K, int ncols, int Nb, const double *Mp,
                    const double *phi_tgt, const int *mon_inv, double *b_out, double *A, cudaStream_t st);
int launch_surface_charges(int nsys, int ndir, int Nb, const double *Bq, const double4_32a *dirs, const double *A,
                           double Rs, double2 *img, cudaStream_t st);
int launch_surface_pairs(const SysDesc *sys, int nsys, int total_items, const long long *ns, const float4 *src_hi,
                         const float4 *src_lo, const double4_32a *src64, int ndir, const double4_32a *dirs,
                         const double2 *img, double Rs, double dr, int precision, double *phi_out,
                         double *e_out, cudaStream_t st);
int launch_series_field(const SysDesc *sys, int nsys, long long max_n, int P, double Rs, const double *norm,
                        const double *A, const float4 *src_hi, const float4 *src_lo, const double4_32a *src64,
                        double *phi_out, double *e_out, cudaStream_t st);
int finalize_blocks(long long max_n);
int launch_finalize(const SysDesc *sys, int nsys, long long max_n, const int *perm, const double *q,
                    const double *phi_tgt, const double *e_part, const double *phi_out, const double *e_out,
                    double *forces, double *pot, long long *owned_idx, double *upart, double *energy, int *status,
                    cudaStream_t st);

// api.cu: free a plan's workspace when it holds more than max_keep bytes
// (used by the serving lanes to stay inside their memory budget).
void plan_trim_workspace(hsma_plan_t plan, size_t max_keep);
// api.cu: allocate a plan's workspace and pinned staging for a batch of nsys
// systems of n_each particles now (so that calls up to that size allocate
// nothing; allocation and freeing synchronise the device)
int plan_reserve(hsma_plan_t plan, int nsys, long long n_each);

// tc_fit.cu: the tensor-core fit.  Mp_hi / Mp_lo: M+ as two BF16 words;
// Mdf: M (K x n_cols) as FP32 word pairs (prepare_tc_operands fills all of
// them at plan time).
int launch_fit_tc(const SysDesc *sys, int nsys, int bc, int K, int ncols, int Nb, const void *Mp_hi,
                  const void *Mp_lo, const void *Mdf, const double *phi_tgt, const int *mon_inv, double *b_out,
                  double *A, float *work, int *status, int sms, cudaStream_t st);
int prepare_tc_operands(int K, int ncols, const double *Mp, const double *Mrow, void *Mp_hi, void *Mp_lo, void *Mdf,
                        cudaStream_t st);
size_t tc_operand_bytes(int K, int ncols);
size_t tc_residual_matrix_bytes(int K, int ncols);
size_t tc_work_bytes(int K, int ncols, int nsys, int sms);

}  // namespace hsma
