// In-set generation (Sec. II.A; Table I "generate images"): the N sources and
// every image with |r| < Rs.  Images follow the periodic sum of Sec. II
// (r_j + k∘L) or, for the grounded box, Eq. "diel" at gamma = -1
// ((-1)^k ∘ r_j + k∘L with charge (-1)^{|k|} q_j).
//
// Four kernels give a deterministic compacted order -- shift k = 0 first (so
// in-set slot i of a system is its i-th particle in spatial order, perm[i]),
// then the other shifts in the order of the shift table, each over the
// particles in spatial order:
//   centre  : per particle (spatial order) the centred, wrapped position and
//             charge, once (the FP64 wrap is not repeated for every shift),
//             an FP32 copy and per-block charge sums;
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

__global__ void __launch_bounds__(kInsetThreads) inset_centre_kernel(InsetArgs a)
{
    __shared__ double red[32];
    int sys_i = blockIdx.y;
    const SysDesc sd = a.sys[sys_i];
    if (blockIdx.x >= sd.nblk) return;
    long long j = (long long)blockIdx.x * kInsetThreads + threadIdx.x;
    double qv = 0.0;
    if (j < sd.n) {
        Centred c = load_centred(a.xyz, a.q, sd.part_off + a.perm[sd.part_off + j], a.g);
        if (!c.ok) atomicOr(&a.status[sys_i], ST_OUT_OF_BOX);
        a.cen[sd.part_off + j] = make_double4_32a(c.x, c.y, c.z, c.q);
        a.cenf[sd.part_off + j] = make_float4((float)c.x, (float)c.y, (float)c.z, 0.f);
        qv = c.q;
    }
    // per-block charge sums for the neutrality check (fixed reduction order)
    const double s = block_sum(qv, red);
    const double sa = block_sum(fabs(qv), red);
    if (threadIdx.x == 0) a.qsums[sd.cnt_off / a.n_shifts + blockIdx.x] = make_double2(s, sa);
}

__device__ __forceinline__ Centred centred_at(const InsetArgs &a, const SysDesc &sd, long long j)
{
    const double4_32a v = a.cen[sd.part_off + j];
    Centred c;
    c.x = v.x;
    c.y = v.y;
    c.z = v.z;
    c.q = v.w;
    c.ok = true;
    return c;
}

// Membership of the image of particle j under a shift: decided in FP32 when
// |r|^2 is clearly inside or outside the sphere, else by the FP64 test of
// image_of (the reference predicate).  Near the sphere each coordinate is
// at most Rs and carries at most three FP32 roundings of terms no larger
// than Rs + max L, so the FP32 |r|^2 is within about 2e-6 (Rs + max L)^2 of
// the exact one; the band, 1e-4 (Rs + max L)^2, is fifty times wider and
// every decision taken in FP32 equals the FP64 one.
__device__ __forceinline__ bool in_set(const InsetArgs &a, const SysDesc &sd, long long j, int4 s)
{
    if (s.x == 0 && s.y == 0 && s.z == 0) return true;
    const float4 c = a.cenf[sd.part_off + j];
    float sx = 1.f, sy = 1.f, sz = 1.f;
    if (a.g.bc == HSMA_BC_GROUNDED) {
        if (s.x & 1) sx = -1.f;
        if (s.y & 1) sy = -1.f;
        if (s.z & 1) sz = -1.f;
    }
    const float x = fmaf(sx, c.x, (float)s.x * (float)a.g.L[0]);
    const float y = fmaf(sy, c.y, (float)s.y * (float)a.g.L[1]);
    const float z = fmaf(sz, c.z, (float)s.z * (float)a.g.L[2]);
    const float r2 = fmaf(x, x, fmaf(y, y, z * z));
    const double lmax = fmax(a.g.L[0], fmax(a.g.L[1], a.g.L[2]));
    const float band = (float)(1e-4 * (a.g.Rs + lmax) * (a.g.Rs + lmax));
    const float rs2 = (float)(a.g.Rs * a.g.Rs);
    if (r2 < rs2 - band) return true;
    if (r2 > rs2 + band) return false;
    double dx, dy, dz, dq;
    return image_of(centred_at(a, sd, j), s, a.g, dx, dy, dz, dq);
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
    if (j < sd.n) hit = in_set(a, sd, j, a.shifts[sh]) ? 1 : 0;
    int cnt = __syncthreads_count(hit);
    if (threadIdx.x == 0) a.counts[sd.cnt_off + (long long)sh * sd.nblk + blk] = cnt;
}

__global__ void __launch_bounds__(1024) inset_scan_kernel(InsetArgs a)
{
    __shared__ int wsum[32];
    __shared__ long long carry;
    __shared__ double red[32];
    int sys_i = blockIdx.x;
    const SysDesc sd = a.sys[sys_i];
    const long long total = block_scan_inplace(a.counts + sd.cnt_off, (long long)a.n_shifts * sd.nblk, wsum, &carry);
    if (threadIdx.x == 0) a.ns[sys_i] = total;
    // neutrality of periodic systems: |sum q| <= 1e-12 sum |q|, from the
    // per-block sums in block order (deterministic)
    double s = 0.0, sa = 0.0;
    const double2 *qs = a.qsums + sd.cnt_off / a.n_shifts;
    for (int b = threadIdx.x; b < sd.nblk; b += blockDim.x) {
        s += qs[b].x;
        sa += qs[b].y;
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
    if (j < sd.n) hit = in_set(a, sd, j, a.shifts[sh]);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned m = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) wsum[wid] = __popc(m);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < wid; ++w) before += wsum[w];
    before += __popc(m & ((1u << lane) - 1u));
    if (!hit) return;
    // the image itself in FP64 (positions of the in-set are exact to FP64)
    double x, y, z, q;
    image_of(centred_at(a, sd, j), a.shifts[sh], a.g, x, y, z, q);
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
    inset_centre_kernel<<<dim3(a.nblk_max, a.nsys), kInsetThreads, 0, st>>>(a);
    HSMA_LAUNCHED();
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
