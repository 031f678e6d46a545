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
#include <algorithm>

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
    if (a.cand) {  // candidate pass: record (spatial index, shift)
        a.cand[sd.src_off + a.counts[sd.cnt_off + (long long)sh * sd.nblk + blk] + before] = make_int2((int)j, sh);
        return;
    }
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

// Regenerate the in-set of a step from a candidate list (see RegenArgs).
// Candidate c is image shift[c.y] of particle perm[c.x].  The particle's
// position u continues the build position by its displacement (periodic:
// the minimum image of the change), so every candidate keeps the lattice
// point it had at the build, moved with its particle: the images of the
// periodic lattice are the same points whichever copy is called the
// particle.  A particle that crossed a wall has u outside the box; its
// canonical position, the one a fresh step evaluates, is w = u - s L with
// the wall shift s.  Its own slot (shift 0, the first n candidates in
// spatial order) takes w, and the candidate of shift -s -- the point w in
// the build's frame, always in the list when the skin is below Rs - R0 --
// takes u, so the point set is unchanged and the particle is evaluated where
// a fresh step evaluates it.  Membership is the FP64 test |r| < Rs of the
// step (shift 0 always in).  A pass per particle computes u and the checks;
// three passes give the compacted in-set in candidate order: count per block
// of candidates, exclusive scan, scatter.
struct RegenPoint {
    double x, y, z, q;
    bool in;
};

// Per particle (spatial order): the continued position u and the charge, and
// the checks (finite, inside a grounded box, moved less than the skin, same
// charge as at the build).
__global__ void __launch_bounds__(kInsetThreads) regen_centre_kernel(RegenArgs r)
{
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < r.n;
         j += (long long)gridDim.x * blockDim.x) {
        const long long i = r.perm[j];
        const double4_32a b = r.x0[j];
        const double b0[3] = {b.x, b.y, b.z};
        double u[3];
        bool ok = true;
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double L = r.g.L[a];
            double v = r.xyz[3 * i + a];
            if (!(v == v) || isinf(v)) ok = false;
            if (r.g.bc == HSMA_BC_GROUNDED && !(v > 0.0 && v < L)) ok = false;
            double d = (v - 0.5 * L) - b0[a];
            if (r.g.bc == HSMA_BC_PERIODIC) d -= L * rint(d / L);
            u[a] = b0[a] + d;
            d2 += d * d;
        }
        const double qi = r.q[i];
        if (!ok || !(qi == qi) || isinf(qi)) atomicOr(r.status, ST_OUT_OF_BOX);
        if (d2 >= r.skin * r.skin || qi != b.w) atomicOr(r.status, ST_STALE);
        r.u[j] = make_double4_32a(u[0], u[1], u[2], qi);
    }
}

__device__ __forceinline__ RegenPoint regen_point(const RegenArgs &r, long long c)
{
    const int2 e = r.cand[c];
    const double4_32a uq = r.u[e.x];
    const double u[3] = {uq.x, uq.y, uq.z};
    int ws[3];
    for (int a = 0; a < 3; ++a)  // wall shift of the continued position (0 inside the box)
        ws[a] = r.g.bc == HSMA_BC_PERIODIC ? (int)floor((u[a] + 0.5 * r.g.L[a]) / r.g.L[a]) : 0;
    const double qi = uq.w;
    int4 s = r.shifts[e.y];
    const bool zero = s.x == 0 && s.y == 0 && s.z == 0;
    const bool crossed = ws[0] | ws[1] | ws[2];
    if (crossed) {
        if (zero) {
            s = make_int4(-ws[0], -ws[1], -ws[2], 0);  // own slot: the canonical position w
        } else if (s.x == -ws[0] && s.y == -ws[1] && s.z == -ws[2]) {
            s = make_int4(0, 0, 0, 0);  // the slot of w in the build's frame: the point u
        }
    }
    double sx = 1.0, sy = 1.0, sz = 1.0;
    RegenPoint pt;
    pt.q = qi;
    if (r.g.bc == HSMA_BC_GROUNDED) {
        if (s.x & 1) sx = -1.0;
        if (s.y & 1) sy = -1.0;
        if (s.z & 1) sz = -1.0;
        if (s.w & 1) pt.q = -pt.q;
    }
    pt.x = sx * u[0] + s.x * r.g.L[0];
    pt.y = sy * u[1] + s.y * r.g.L[1];
    pt.z = sz * u[2] + s.z * r.g.L[2];
    pt.in = zero || pt.x * pt.x + pt.y * pt.y + pt.z * pt.z < r.g.Rs * r.g.Rs;
    return pt;
}

__global__ void __launch_bounds__(kInsetThreads) regen_count_kernel(RegenArgs r)
{
    const long long nc = min(*r.ncand, r.cap_cand);
    const long long nblk = (nc + kInsetThreads - 1) / kInsetThreads;
    for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const long long c = blk * kInsetThreads + threadIdx.x;
        int hit = 0;
        if (c < nc) hit = regen_point(r, c).in ? 1 : 0;
        const int cnt = __syncthreads_count(hit);
        if (threadIdx.x == 0) r.counts[blk] = cnt;
    }
}

__global__ void __launch_bounds__(1024) regen_scan_kernel(RegenArgs r)
{
    __shared__ int wsum[32];
    __shared__ long long carry;
    const long long nc = min(*r.ncand, r.cap_cand);
    const long long nblk = (nc + kInsetThreads - 1) / kInsetThreads;
    const long long total = block_scan_inplace(r.counts, nblk, wsum, &carry);
    if (threadIdx.x == 0) {
        r.ns[0] = min(total, r.cap);
        if (total > r.cap) atomicOr(r.status, ST_STALE);  // more members than in-set slots: rebuild
    }
}

__global__ void __launch_bounds__(kInsetThreads) regen_scatter_kernel(RegenArgs r)
{
    __shared__ int wsum[kInsetThreads / 32];
    const long long nc = min(*r.ncand, r.cap_cand);
    const long long nblk = (nc + kInsetThreads - 1) / kInsetThreads;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const long long c = blk * kInsetThreads + threadIdx.x;
        RegenPoint pt;
        pt.in = false;
        if (c < nc) pt = regen_point(r, c);
        const unsigned m = __ballot_sync(0xffffffffu, pt.in);
        __syncthreads();  // wsum of the previous block is read
        if (lane == 0) wsum[wid] = __popc(m);
        __syncthreads();
        int before = 0;
        for (int w = 0; w < wid; ++w) before += wsum[w];
        before += __popc(m & ((1u << lane) - 1u));
        const long long slot = r.counts[blk] + before;
        if (!pt.in || slot >= r.cap) continue;
        if (r.src64) r.src64[slot] = make_double4_32a(pt.x, pt.y, pt.z, pt.q);
        if (r.src_hi) {
            float hx, lx, hy, ly, hz, lz;
            split_f64(pt.x, hx, lx);
            split_f64(pt.y, hy, ly);
            split_f64(pt.z, hz, lz);
            r.src_hi[slot] = make_float4(hx, hy, hz, (float)pt.q);
            r.src_lo[slot] = make_float4(lx, ly, lz, 0.f);
        }
    }
}

}  // namespace

int launch_inset_candidates(const InsetArgs &a, cudaStream_t st)
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

int launch_inset_regen(const RegenArgs &r, cudaStream_t st)
{
    const long long nblk = (r.cap_cand + kInsetThreads - 1) / kInsetThreads;
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(nblk, 1LL << 14));
    const unsigned pgrid = (unsigned)std::max<long long>(1, std::min<long long>((r.n + kInsetThreads - 1) / kInsetThreads, 1LL << 14));
    regen_centre_kernel<<<pgrid, kInsetThreads, 0, st>>>(r);
    HSMA_LAUNCHED();
    regen_count_kernel<<<grid, kInsetThreads, 0, st>>>(r);
    HSMA_LAUNCHED();
    regen_scan_kernel<<<1, 1024, 0, st>>>(r);
    HSMA_LAUNCHED();
    regen_scatter_kernel<<<grid, kInsetThreads, 0, st>>>(r);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

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
