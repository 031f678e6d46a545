// Spatial order of the particles and bounding boxes of source tiles.
//
// The particles of each system are put in Morton order of a G^3 grid over the
// box (G = 2^gbits cells per axis) by a stable LSD radix sort on 8-bit digits
// (key ties keep the input order, so the result is deterministic).  The in-set
// is then generated in (shift, sorted particle) order, which makes every run
// of consecutive in-set entries -- a shared-memory tile of sources, or a block
// of target particles -- a compact piece of space.  tile_boxes_kernel records
// the axis-aligned box of every tile; the pair kernel uses the distance
// between a target block's box and a tile's box to decide whether the tile
// needs the split-word differences (see pair.cu).
#include "common.cuh"

namespace hsma {

namespace {

constexpr int kSortThreads = 256;  // elements per sort block (= in-set block size)
constexpr int kRadix = 256;

__device__ __forceinline__ unsigned spread3(unsigned v)
{
    // bits b0 b1 b2 ... -> b0 . . b1 . . b2 (for up to 10 input bits)
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void __launch_bounds__(kSortThreads) morton_keys_kernel(SortArgs a)
{
    const int s = blockIdx.y;
    const SysDesc sd = a.sys[s];
    long long j = (long long)blockIdx.x * kSortThreads + threadIdx.x;
    if (blockIdx.x >= sd.nblk || j >= sd.n) return;
    const int G = 1 << sd.gbits;
    const double *p = a.xyz + 3 * (sd.part_off + j);
    unsigned c[3];
    for (int ax = 0; ax < 3; ++ax) {
        double L = a.g.L[ax];
        double v = p[ax];
        if (a.g.bc == HSMA_BC_PERIODIC) v = v - floor(v / L) * L;
        double f = v / L * G;
        int ci = (f == f) ? (int)floor(f) : 0;
        ci = ci < 0 ? 0 : (ci >= G ? G - 1 : ci);
        c[ax] = (unsigned)ci;
    }
    a.keys[sd.part_off + j] = (int)(spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2));
    a.vals[sd.part_off + j] = (int)j;
}

// Per (system, block): histogram of the current digit, stored digit-major.
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(SortArgs a, const int *keys, int shift)
{
    __shared__ int h[kRadix];
    const int s = blockIdx.y;
    const SysDesc sd = a.sys[s];
    if (blockIdx.x >= sd.nblk) return;
    h[threadIdx.x] = 0;
    __syncthreads();
    long long j = (long long)blockIdx.x * kSortThreads + threadIdx.x;
    if (j < sd.n) atomicAdd(&h[(keys[sd.part_off + j] >> shift) & (kRadix - 1)], 1);
    __syncthreads();
    a.hist[sd.hist_off + (long long)threadIdx.x * sd.nblk + blockIdx.x] = h[threadIdx.x];
}

// Per system: exclusive prefix over (digit, block) in digit-major order.
__global__ void __launch_bounds__(1024) radix_scan_kernel(SortArgs a)
{
    __shared__ int wsum[32];
    __shared__ long long carry;
    const SysDesc sd = a.sys[blockIdx.x];
    block_scan_inplace(a.hist + sd.hist_off, (long long)kRadix * sd.nblk, wsum, &carry);
}

// Stable scatter of one digit pass: the rank of an element among equal digits
// of its block is (equal digits in earlier warps) + (equal digits in earlier
// lanes of its warp).
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(SortArgs a, const int *kin, const int *vin,
                                                                     int *kout, int *vout, int shift)
{
    constexpr int kWarps = kSortThreads / 32;
    __shared__ int wcount[kWarps][kRadix];
    const int s = blockIdx.y;
    const SysDesc sd = a.sys[s];
    if (blockIdx.x >= sd.nblk) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kSortThreads) (&wcount[0][0])[i] = 0;
    __syncthreads();
    long long j = (long long)blockIdx.x * kSortThreads + threadIdx.x;
    const bool valid = j < sd.n;
    int key = valid ? kin[sd.part_off + j] : 0;
    int val = valid ? vin[sd.part_off + j] : 0;
    int d = valid ? ((key >> shift) & (kRadix - 1)) : -1;
    unsigned same = __match_any_sync(0xffffffffu, d);
    int rank = __popc(same & ((1u << lane) - 1u));
    int leader = __ffs(same) - 1;
    if (valid && lane == leader) wcount[wid][d] = __popc(same);
    __syncthreads();
    if (!valid) return;
    int before = 0;
    for (int w = 0; w < wid; ++w) before += wcount[w][d];
    long long dst = sd.part_off + a.hist[sd.hist_off + (long long)d * sd.nblk + blockIdx.x] + before + rank;
    kout[dst] = key;
    vout[dst] = val;
}

// Axis-aligned box of every tile of `tile` consecutive in-set entries (high
// FP32 words), widened by a relative margin that covers the low words.
__global__ void tile_boxes_kernel(const SysDesc *sys, const long long *ns, const float4 *src_hi, int tile,
                                  float4 *boxes)
{
    const int s = blockIdx.y;
    const SysDesc sd = sys[s];
    const long long Ns = ns[s];
    const long long ntiles = (Ns + tile - 1) / tile;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= ntiles) return;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    long long b0 = (long long)warp * tile;
    long long b1 = min(b0 + tile, Ns);
    for (long long i = b0 + lane; i < b1; i += 32) {
        float4 p = src_hi[sd.src_off + i];
        lo[0] = fminf(lo[0], p.x); hi[0] = fmaxf(hi[0], p.x);
        lo[1] = fminf(lo[1], p.y); hi[1] = fmaxf(hi[1], p.y);
        lo[2] = fminf(lo[2], p.z); hi[2] = fmaxf(hi[2], p.z);
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int ax = 0; ax < 3; ++ax) {
            lo[ax] = fminf(lo[ax], __shfl_xor_sync(0xffffffffu, lo[ax], o));
            hi[ax] = fmaxf(hi[ax], __shfl_xor_sync(0xffffffffu, hi[ax], o));
        }
    if (lane == 0) {
        const float m = 1e-6f;
        float4 *b = boxes + 2 * (sd.tile_off + warp);
        b[0] = make_float4(lo[0] - m * fabsf(lo[0]) - 1e-30f, lo[1] - m * fabsf(lo[1]) - 1e-30f,
                           lo[2] - m * fabsf(lo[2]) - 1e-30f, 0.f);
        b[1] = make_float4(hi[0] + m * fabsf(hi[0]) + 1e-30f, hi[1] + m * fabsf(hi[1]) + 1e-30f,
                           hi[2] + m * fabsf(hi[2]) + 1e-30f, 0.f);
    }
}

}  // namespace

int launch_sort_particles(const SortArgs &a, int nblk_max, cudaStream_t st)
{
    dim3 grid(nblk_max, a.nsys);
    morton_keys_kernel<<<grid, kSortThreads, 0, st>>>(a);
    HSMA_LAUNCHED();
    int *kin = a.keys, *vin = a.vals, *kout = a.keys2, *vout = a.vals2;
    for (int pass = 0; pass < 2; ++pass) {
        const int shift = 8 * pass;
        radix_hist_kernel<<<grid, kSortThreads, 0, st>>>(a, kin, shift);
        HSMA_LAUNCHED();
        radix_scan_kernel<<<a.nsys, 1024, 0, st>>>(a);
        HSMA_LAUNCHED();
        radix_scatter_kernel<<<grid, kSortThreads, 0, st>>>(a, kin, vin, kout, vout, shift);
        HSMA_LAUNCHED();
        int *t = kin; kin = kout; kout = t;
        t = vin; vin = vout; vout = t;
    }
    // after two passes the sorted order is back in keys/vals (a.vals = perm)
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

int launch_tile_boxes(const SysDesc *sys, int nsys, long long max_tiles, const long long *ns, const float4 *src_hi,
                      int tile, float4 *boxes, cudaStream_t st)
{
    dim3 grid((unsigned)((max_tiles * 32 + 255) / 256), nsys);
    tile_boxes_kernel<<<grid, 256, 0, st>>>(sys, ns, src_hi, tile, boxes);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

}  // namespace hsma

namespace hsma {

namespace {

// out[k] = in[perm[k]] for the three monitoring-target arrays.
__global__ void gather_targets_kernel(int n, const int *perm, const double4_32a *in64, const float4 *inhi,
                                      const float4 *inlo, double4_32a *out64, float4 *outhi, float4 *outlo)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int i = perm[k];
    out64[k] = in64[i];
    outhi[k] = inhi[i];
    outlo[k] = inlo[i];
}

// Box of every run of `block` consecutive points of an array (high words,
// widened like the tile boxes).
__global__ void array_boxes_kernel(int n, const float4 *hi, int block, float4 *boxes)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nb = (n + block - 1) / block;
    if (warp >= nb) return;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hh[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = warp * block + lane; i < min(n, (warp + 1) * block); i += 32) {
        float4 p = hi[i];
        lo[0] = fminf(lo[0], p.x); hh[0] = fmaxf(hh[0], p.x);
        lo[1] = fminf(lo[1], p.y); hh[1] = fmaxf(hh[1], p.y);
        lo[2] = fminf(lo[2], p.z); hh[2] = fmaxf(hh[2], p.z);
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int ax = 0; ax < 3; ++ax) {
            lo[ax] = fminf(lo[ax], __shfl_xor_sync(0xffffffffu, lo[ax], o));
            hh[ax] = fmaxf(hh[ax], __shfl_xor_sync(0xffffffffu, hh[ax], o));
        }
    if (lane == 0) {
        const float m = 1e-6f;
        boxes[2 * warp] = make_float4(lo[0] - m * fabsf(lo[0]) - 1e-30f, lo[1] - m * fabsf(lo[1]) - 1e-30f,
                                      lo[2] - m * fabsf(lo[2]) - 1e-30f, 0.f);
        boxes[2 * warp + 1] = make_float4(hh[0] + m * fabsf(hh[0]) + 1e-30f, hh[1] + m * fabsf(hh[1]) + 1e-30f,
                                          hh[2] + m * fabsf(hh[2]) + 1e-30f, 0.f);
    }
}

}  // namespace

int launch_gather_targets(int n, const int *perm, const double4_32a *in64, const float4 *inhi, const float4 *inlo,
                          double4_32a *out64, float4 *outhi, float4 *outlo, cudaStream_t st)
{
    gather_targets_kernel<<<(n + 127) / 128, 128, 0, st>>>(n, perm, in64, inhi, inlo, out64, outhi, outlo);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

int launch_array_boxes(int n, const float4 *hi, int block, float4 *boxes, cudaStream_t st)
{
    int nb = (n + block - 1) / block;
    array_boxes_kernel<<<(nb * 32 + 127) / 128, 128, 0, st>>>(n, hi, block, boxes);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

}  // namespace hsma
