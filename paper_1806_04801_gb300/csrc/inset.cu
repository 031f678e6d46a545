// In-set generation (Sec. II.A; Table I "generate images"): the N sources and
// every image with |r| < Rs.  Images follow the periodic sum of Sec. II
// (r_j + k∘L) or, for the grounded box, Eq. "diel" at gamma = -1
// ((-1)^k ∘ r_j + k∘L with charge (-1)^{|k|} q_j).
//
// Three kernels give a deterministic compacted order -- shift k = 0 first (so
// in-set slot i of a system is its i-th particle in spatial order, perm[i]),
// then the other shifts in the order of the shift table, each over the
// particles in spatial order:
//   count   : per (system, shift, block of particles) the number of hits;
//   scan    : per system, exclusive prefix over (shift, block) + totals, and
//             the neutrality check of periodic systems;
//   scatter : re-evaluates the predicate and writes each hit to its slot.
#include "common.cuh"

namespace hsma {

namespace {

constexpr int kInsetThreads = 256;

struct Centred {
    double x, y, z, q;
    bool ok;
};

// Box frame -> centred frame; periodic inputs are wrapped into [0, L) first.
__device__ __forceinline__ Centred load_centred(const double *xyz, const double *q, long long i, const Geometry &g)
{
    Centred c;
    double p[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
    c.ok = true;
    for (int a = 0; a < 3; ++a) {
        double L = g.L[a];
        double v = p[a];
        if (!(v == v) || isinf(v)) c.ok = false;
        if (g.bc == HSMA_BC_PERIODIC) {
            v = v - floor(v / L) * L;
        } else if (!(v > 0.0 && v < L)) {
            c.ok = false;
        }
        p[a] = v - 0.5 * L;
    }
    c.x = p[0];
    c.y = p[1];
    c.z = p[2];
    c.q = q[i];
    if (!(c.q == c.q) || isinf(c.q)) c.ok = false;
    return c;
}

// Image of source c under shift s (kx, ky, kz, |k| parity in .w).
__device__ __forceinline__ bool image_of(const Centred &c, int4 s, const Geometry &g, double &x, double &y,
                                         double &z, double &q)
{
    double sx = 1.0, sy = 1.0, sz = 1.0;
    q = c.q;
    if (g.bc == HSMA_BC_GROUNDED) {
        if (s.x & 1) sx = -1.0;
        if (s.y & 1) sy = -1.0;
        if (s.z & 1) sz = -1.0;
        if (s.w & 1) q = -q;
    }
    x = sx * c.x + s.x * g.L[0];
    y = sy * c.y + s.y * g.L[1];
    z = sz * c.z + s.z * g.L[2];
    if (s.x == 0 && s.y == 0 && s.z == 0) return true;
    return x * x + y * y + z * z < g.Rs * g.Rs;
}

__global__ void __launch_bounds__(kInsetThreads) inset_count_kernel(InsetArgs a)
{
    int sys_i = blockIdx.z;
    const SysDesc sd = a.sys[sys_i];
    int blk = blockIdx.x;
    if (blk >= sd.nblk) return;
    int sh = blockIdx.y;
    long long j = (long long)blk * kInsetThreads + threadIdx.x;
    int hit = 0;
    if (j < sd.n) {
        Centred c = load_centred(a.xyz, a.q, sd.part_off + a.perm[sd.part_off + j], a.g);
        if (sh == 0 && !c.ok) atomicOr(&a.status[sys_i], ST_OUT_OF_BOX);
        double x, y, z, q;
        hit = image_of(c, a.shifts[sh], a.g, x, y, z, q) ? 1 : 0;
    }
    int cnt = __syncthreads_count(hit);
    if (threadIdx.x == 0) a.counts[sd.cnt_off + (long long)sh * sd.nblk + blk] = cnt;
}

__global__ void __launch_bounds__(1024) inset_scan_kernel(InsetArgs a)
{
    __shared__ int wsum[32];
    __shared__ int carry;
    __shared__ double red[32];
    int sys_i = blockIdx.x;
    const SysDesc sd = a.sys[sys_i];
    long long total = (long long)a.n_shifts * sd.nblk;
    int *cnt = a.counts + sd.cnt_off;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long base = 0; base < total; base += blockDim.x) {
        long long t = base + threadIdx.x;
        int v = (t < total) ? cnt[t] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int w = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
            int wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                int u = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += u;
            }
            wsum[lane] = wi - w;  // exclusive prefix of warp sums
        }
        __syncthreads();
        int excl = carry + wsum[wid] + incl - v;
        if (t < total) cnt[t] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.ns[sys_i] = carry;
    // neutrality of periodic systems: |sum q| <= 1e-12 sum |q| (deterministic order)
    double s = 0.0, sa = 0.0;
    for (long long j = threadIdx.x; j < sd.n; j += blockDim.x) {
        double qq = a.q[sd.part_off + j];
        s += qq;
        sa += fabs(qq);
    }
    s = block_sum(s, red);
    sa = block_sum(sa, red);
    if (threadIdx.x == 0 && a.g.bc == HSMA_BC_PERIODIC && fabs(s) > 1e-12 * sa)
        atomicOr(&a.status[sys_i], ST_NONNEUTRAL);
}

__global__ void __launch_bounds__(kInsetThreads) inset_scatter_kernel(InsetArgs a)
{
    __shared__ int wsum[kInsetThreads / 32];
    int sys_i = blockIdx.z;
    const SysDesc sd = a.sys[sys_i];
    int blk = blockIdx.x;
    if (blk >= sd.nblk) return;
    int sh = blockIdx.y;
    long long j = (long long)blk * kInsetThreads + threadIdx.x;
    bool hit = false;
    double x = 0, y = 0, z = 0, q = 0;
    if (j < sd.n) {
        Centred c = load_centred(a.xyz, a.q, sd.part_off + a.perm[sd.part_off + j], a.g);
        hit = image_of(c, a.shifts[sh], a.g, x, y, z, q);
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned m = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) wsum[wid] = __popc(m);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < wid; ++w) before += wsum[w];
    before += __popc(m & ((1u << lane) - 1u));
    if (!hit) return;
    long long slot = sd.src_off + a.counts[sd.cnt_off + (long long)sh * sd.nblk + blk] + before;
    if (a.src64) a.src64[slot] = make_double4_32a(x, y, z, q);
    if (a.src_hi) {
        float hx, lx, hy, ly, hz, lz;
        split_f64(x, hx, lx);
        split_f64(y, hy, ly);
        split_f64(z, hz, lz);
        a.src_hi[slot] = make_float4(hx, hy, hz, (float)q);
        a.src_lo[slot] = make_float4(lx, ly, lz, 0.f);
    }
}

}  // namespace

int launch_inset(const InsetArgs &a, cudaStream_t st)
{
    dim3 grid(a.nblk_max, a.n_shifts, a.nsys);
    inset_count_kernel<<<grid, kInsetThreads, 0, st>>>(a);
    HSMA_LAUNCHED();
    inset_scan_kernel<<<a.nsys, 1024, 0, st>>>(a);
    HSMA_LAUNCHED();
    inset_scatter_kernel<<<grid, kInsetThreads, 0, st>>>(a);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

}  // namespace hsma
