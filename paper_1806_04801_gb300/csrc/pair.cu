// Near-field Coulomb sums (Sec. II.A: Phi_in = sum_{j <= N_s} q_j/|r_j - r|,
// evaluated at the particles -- potential and field -- and at the monitoring
// points -- potential).  This is the hot loop of the method (Sec. II.C: "the
// most time-consuming calculations").
//
// Work decomposition: one persistent grid pulls items (system, target block,
// source chunk) from an atomic counter (or, in the one-item mode of serving
// lanes, CTA b does item b and exits, so that higher-priority work on other
// streams gets SMs between items).  A CTA stages the chunk's sources in
// shared-memory tiles with 1-D bulk copies (cp.async.bulk, completion on an
// mbarrier, two buffers in flight) and every thread sums the tile into the
// registers of its T targets.  Each item writes one partial record per target;
// a second kernel adds the chunks of every target in a fixed order, so results
// do not depend on scheduling.
//
// FP32 form: positions are held as two FP32 words (hi + lo, the in-set kernel
// splits the FP64 value), so the difference (y_hi - x_hi) + (y_lo - x_lo) is
// accurate to a few FP32 ulps of the distance itself, even for the closest
// pairs; 1/r comes from the SFU (rsqrt.approx); the potential is summed in
// FP32 over 32 sources and the field over a whole tile, then folded into
// double-float (hi, lo) accumulators with an error-free TwoSum.  The packed
// variants run the same arithmetic on two sources per f32x2 instruction
// (fma/add/mul.rn.f32x2), which halves the issue slots of the FP32 work.
//
// FP64 form: the same loop in double, rsqrt() from the CUDA math library.
#include "common.cuh"

namespace hsma {

namespace {

constexpr int kThreads = 128;
// FP32 form: T targets per thread (T = 2, 3 or 4, by variant); a block of
// 128 T targets is exactly one in-set tile of 128 T sources, so a particle
// block's box is its tile's box.
constexpr int kT64 = 2;
constexpr int kTB64 = kThreads * kT64;
constexpr int kTile64 = 256;
constexpr int kFold = 32;               // potential fold interval (sources)
constexpr int kFold2 = 64;              // packed loop: 32 sources per lane
constexpr bool kCpDouble = true;        // mode 1: two interleaved buffers, one barrier per tile
constexpr float kFar = 1.0e4f;          // position of zero-charge padding sources

struct Item {
    int sys, tb, chunk;
};

__device__ __forceinline__ Item decode_item(const PairArgs &a, int item)
{
    int lo = 0, hi = a.nsys - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (a.sys[mid].item_off <= item)
            lo = mid;
        else
            hi = mid - 1;
    }
    const SysDesc &sd = a.sys[lo];
    int local = item - sd.item_off;
    Item it;
    it.sys = lo;
    it.chunk = local / sd.ntb;
    it.tb = local - it.chunk * sd.ntb;
    return it;
}

// ------------------------------------------------------------ FP32 tiles
// SKIP: 0 = no exclusion; 1 = skip the target's own slot (self_rel[t] = own
// slot - tile start); 2 = skip pairs at distance exactly zero.
// SPLIT: use the low words of both positions in the difference.  A tile whose
// box is at least `far` away from the target block's box uses the high words
// only: their rounding (<= 2^-24 |x|) then changes each distance by a relative
// ~1e-6 or less, while the closest pairs -- where an absolute error of
// ~1e-7 would matter -- always take the split form.
template <int T, int UNROLL, bool FIELD, int SKIP, bool SPLIT>
__device__ __forceinline__ void tile32(const float4 *__restrict__ sh, const float4 *__restrict__ sl, int cnt_pad,
                                       const float (&th)[T][3], const float (&tl)[T][3],
                                       const int (&self_rel)[T], float2 (&phi)[T], float2 (&g)[T][3])
{
    float ga[T][3];
#pragma unroll
    for (int t = 0; t < T; ++t) ga[t][0] = ga[t][1] = ga[t][2] = 0.f;
    for (int s0 = 0; s0 < cnt_pad; s0 += kFold) {
        float pa[T];
#pragma unroll
        for (int t = 0; t < T; ++t) pa[t] = 0.f;
#pragma unroll UNROLL
        for (int s = 0; s < kFold; ++s) {
            const float4 h = sh[s0 + s];
            const float4 l = SPLIT ? sl[s0 + s] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int t = 0; t < T; ++t) {
                float dx, dy, dz;
                if (SPLIT) {
                    dx = (h.x - th[t][0]) + (l.x - tl[t][0]);
                    dy = (h.y - th[t][1]) + (l.y - tl[t][1]);
                    dz = (h.z - th[t][2]) + (l.z - tl[t][2]);
                } else {
                    dx = h.x - th[t][0];
                    dy = h.y - th[t][1];
                    dz = h.z - th[t][2];
                }
                float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                float ri = rsqrt_sfu(r2);
                if (SKIP == 1) ri = (s0 + s == self_rel[t]) ? 0.f : ri;
                if (SKIP == 2) ri = (r2 > 0.f) ? ri : 0.f;
                float qr = h.w * ri;
                pa[t] += qr;
                if (FIELD) {
                    float qr3 = qr * ri * ri;
                    ga[t][0] = fmaf(qr3, dx, ga[t][0]);
                    ga[t][1] = fmaf(qr3, dy, ga[t][1]);
                    ga[t][2] = fmaf(qr3, dz, ga[t][2]);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) phi[t] = df_add(phi[t], pa[t]);
    }
    if (FIELD) {
#pragma unroll
        for (int t = 0; t < T; ++t) {
            g[t][0] = df_add(g[t][0], ga[t][0]);
            g[t][1] = df_add(g[t][1], ga[t][1]);
            g[t][2] = df_add(g[t][2], ga[t][2]);
        }
    }
}

// Packed form of tile32 for two sources at a time (f32x2 instructions: one
// issue slot for two lanes of FP32 work).  The tile is pair-interleaved:
// ph[2p] = (x_2p, x_2p+1, y_2p, y_2p+1), ph[2p+1] = (z_2p, z_2p+1, q_2p, q_2p+1),
// the same for the low words in pl; nth / ntl hold the negated target words
// twice.  Each lane does the operations of tile32 in the same order, except
// that the potential takes q/r with one fused multiply-add.  A lane sums 32
// sources of a 64-source fold interval (even and odd slots), the same FP32
// run length as tile32; the two lane sums are added and folded with one
// TwoSum.  SACC: the double-float accumulators live in shared memory
// (acc[j * kThreads], j = t for the potential of target t, T + 3t + c for
// field component c) instead of phi / g, which frees their registers.
template <int T, int UNROLL, bool FIELD, int SKIP, bool SPLIT, bool SACC>
__device__ __forceinline__ void tile32x2(const float4 *ph, const float4 *pl, int cnt_pad,
                                         const float2 (&nth)[T][3], const float2 (&ntl)[T][3],
                                         const int (&self_rel)[T], float2 (&phi)[T], float2 (&g)[T][3],
                                         float2 *acc)
{
    float2 ga[T][3];
#pragma unroll
    for (int t = 0; t < T; ++t) ga[t][0] = ga[t][1] = ga[t][2] = make_float2(0.f, 0.f);
    for (int s0 = 0; s0 < cnt_pad; s0 += kFold2) {
        float2 pa[T];
#pragma unroll
        for (int t = 0; t < T; ++t) pa[t] = make_float2(0.f, 0.f);
#pragma unroll UNROLL
        for (int s = 0; s < kFold2; s += 2) {
            const float4 a = ph[s0 + s], b = ph[s0 + s + 1];
            const float2 sx = make_float2(a.x, a.y), sy = make_float2(a.z, a.w);
            const float2 sz = make_float2(b.x, b.y), sq = make_float2(b.z, b.w);
            float2 lx = make_float2(0.f, 0.f), ly = lx, lz = lx;
            if (SPLIT) {
                const float4 c = pl[s0 + s], d = pl[s0 + s + 1];
                lx = make_float2(c.x, c.y);
                ly = make_float2(c.z, c.w);
                lz = make_float2(d.x, d.y);
            }
#pragma unroll
            for (int t = 0; t < T; ++t) {
                float2 dx, dy, dz;
                if (SPLIT) {
                    dx = __fadd2_rn(__fadd2_rn(sx, nth[t][0]), __fadd2_rn(lx, ntl[t][0]));
                    dy = __fadd2_rn(__fadd2_rn(sy, nth[t][1]), __fadd2_rn(ly, ntl[t][1]));
                    dz = __fadd2_rn(__fadd2_rn(sz, nth[t][2]), __fadd2_rn(lz, ntl[t][2]));
                } else {
                    dx = __fadd2_rn(sx, nth[t][0]);
                    dy = __fadd2_rn(sy, nth[t][1]);
                    dz = __fadd2_rn(sz, nth[t][2]);
                }
                const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                float2 ri = make_float2(rsqrt_sfu(r2.x), rsqrt_sfu(r2.y));
                if (SKIP == 1) {
                    ri.x = (s0 + s == self_rel[t]) ? 0.f : ri.x;
                    ri.y = (s0 + s + 1 == self_rel[t]) ? 0.f : ri.y;
                }
                if (SKIP == 2) {
                    ri.x = (r2.x > 0.f) ? ri.x : 0.f;
                    ri.y = (r2.y > 0.f) ? ri.y : 0.f;
                }
                pa[t] = __ffma2_rn(sq, ri, pa[t]);
                if (FIELD) {
                    const float2 qr3 = __fmul2_rn(__fmul2_rn(__fmul2_rn(sq, ri), ri), ri);
                    ga[t][0] = __ffma2_rn(qr3, dx, ga[t][0]);
                    ga[t][1] = __ffma2_rn(qr3, dy, ga[t][1]);
                    ga[t][2] = __ffma2_rn(qr3, dz, ga[t][2]);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            if (SACC)
                acc[t * kThreads] = df_add(acc[t * kThreads], pa[t].x + pa[t].y);
            else
                phi[t] = df_add(phi[t], pa[t].x + pa[t].y);
        }
    }
    if (FIELD) {
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (SACC) {
                    float2 &e = acc[(T + 3 * t + c) * kThreads];
                    e = df_add(e, ga[t][c].x + ga[t][c].y);
                } else {
                    g[t][c] = df_add(g[t][c], ga[t][c].x + ga[t][c].y);
                }
            }
    }
}

// Pair-interleave a staged tile (one float4 per source) into the layout of
// tile32x2; slots cnt..cnt_pad-1 become the padding source `pad`.  dst may be
// src: each thread reads both sources of a pair before it rewrites the same
// 32 bytes.
__device__ __forceinline__ void interleave_pairs(const float4 *src, float4 *dst, int cnt, int cnt_pad, float4 pad,
                                                 int tid)
{
    for (int p = tid; 2 * p < cnt_pad; p += kThreads) {
        const int i = 2 * p;
        const float4 a = i < cnt ? src[i] : pad;
        const float4 b = i + 1 < cnt ? src[i + 1] : pad;
        dst[i] = make_float4(a.x, b.x, a.y, b.y);
        dst[i + 1] = make_float4(a.z, b.z, a.w, b.w);
    }
}

// MINB: CTAs per SM the register allocation must allow.  MODE 0: scalar loop
// (tile32); 1: packed two-source loop (tile32x2) on a pair-interleaved copy of
// each staged tile in a third buffer, the staging buffer refilled at once;
// 2: packed loop on the staging buffer interleaved in place, double-float
// accumulators in shared memory (fewer registers, refill after the tile).
// The autotuner picks among these variants.
template <int T, int MINB, int MODE>
__global__ void __launch_bounds__(kThreads, MINB) pair_fp32_kernel(PairArgs a)
{
    constexpr bool X2 = MODE != 0;
    constexpr bool SACC = MODE == 2;
    // source-loop unrolling per variant (measured: 4 targets at 4 CTAs/SM
    // prefers 4, at 5 CTAs/SM 8, two targets a full unroll)
    // (packed: 32 pair steps per fold, unrolled fully for two targets and by
    // half for three and four)
    constexpr int UNROLL = X2 ? (T == 2 ? kFold2 / 2 : kFold2 / 4) : (T == 2 ? kFold : (MINB >= 5 ? 8 : 4));
    constexpr int TB = kThreads * T;  // targets per block
    constexpr int TILE = TB;          // sources per tile
    extern __shared__ __align__(128) float4 smem32[];
    float4 *sh_hi = smem32;                // [2][TILE] staging (bulk copies land here)
    float4 *sh_lo = smem32 + 2 * TILE;  // [2][TILE]
    float4 *cp_hi = smem32 + 4 * TILE;  // MODE 1: [1 or 2][TILE] pair-interleaved tile
    float4 *cp_lo = smem32 + (kCpDouble ? 6 : 5) * TILE;  // MODE 1: [1 or 2][TILE]
    // MODE 2: [4T][kThreads] double-float accumulators, this thread's column
    float2 *acc = reinterpret_cast<float2 *>(smem32 + 4 * TILE) + threadIdx.x;
    __shared__ __align__(8) uint64_t bar[3];
    __shared__ int s_item, s_abort;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        mbar_fence_init();
        s_abort = 0;
    }
    __syncthreads();
    uint32_t parity[2] = {0u, 0u};
    if (a.stall_test) {
        // Test of the bounded-wait path: bar[2] never completes a phase (no
        // arrival, no copy), so the wait runs out after ~1e6 cycles, the
        // status records a timeout and the CTA returns.
        if (!mbar_wait_bounded(&bar[2], 0u, 1000000LL)) atomicOr(&a.status[0], ST_TIMEOUT);
        return;
    }

    for (int round = 0;; ++round) {
        if (tid == 0) s_item = a.one_item ? (round == 0 ? (int)blockIdx.x : a.total_items) : atomicAdd(a.next_item, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.total_items || s_abort) break;
        const Item it = decode_item(a, item);
        const SysDesc sd = a.sys[it.sys];
        const long long Ns = a.ns[it.sys];
        const long long ntiles = (Ns + TILE - 1) / TILE;
        const int t0 = (int)(it.chunk * ntiles / sd.nchunks);
        const int t1 = (int)((it.chunk + 1) * ntiles / sd.nchunks);
        const bool part = it.tb < sd.ntb_part;
        const bool field = part || a.ext_field;
        const long long ntgt = sd.n + a.n_ext;
        // global block index: particle blocks from pb_lo, external from mb_lo
        const int gb = part ? sd.pb_lo + it.tb : sd.mb_lo + it.tb - sd.ntb_part;

        // targets of this thread
        float th[T][3], tl[T][3];
        long long tidx[T];
        long long tb_lo = 0, tb_hi = 0;  // in-set slots of this block's own particles
        if (part) {
            tb_lo = (long long)gb * TB;
            tb_hi = tb_lo + TB;
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            long long k = (long long)gb * TB + t * kThreads + tid;
            bool valid = part ? (k < sd.n) : (k < a.n_ext);
            float4 h = make_float4(kFar, kFar, kFar, 0.f), l = make_float4(0.f, 0.f, 0.f, 0.f);
            if (valid) {
                if (part) {
                    h = a.src_hi[sd.src_off + k];
                    l = a.src_lo[sd.src_off + k];
                } else {
                    h = a.ext_hi[k];
                    l = a.ext_lo[k];
                }
            }
            th[t][0] = h.x; th[t][1] = h.y; th[t][2] = h.z;
            tl[t][0] = l.x; tl[t][1] = l.y; tl[t][2] = l.z;
            tidx[t] = valid ? (part ? k : sd.n + k) : -1;
        }
        float2 nth[T][3], ntl[T][3];  // X2: negated target words, both lanes
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                nth[t][c] = make_float2(-th[t][c], -th[t][c]);
                ntl[t][c] = make_float2(-tl[t][c], -tl[t][c]);
            }
        float2 phi[T], g[T][3];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            phi[t] = make_float2(0.f, 0.f);
            g[t][0] = g[t][1] = g[t][2] = make_float2(0.f, 0.f);
        }
        if constexpr (SACC) {
#pragma unroll
            for (int j = 0; j < 4 * T; ++j) acc[j * kThreads] = make_float2(0.f, 0.f);
        }

        // box of this block's targets (= in-set tile `tb`, its particles), for
        // the near/far decision per source tile
        const bool use_boxes = a.boxes != nullptr && (part || a.ext_boxes != nullptr);
        float4 blo = make_float4(0.f, 0.f, 0.f, 0.f), bhi = blo;
        if (use_boxes) {
            const float4 *bb = part ? a.boxes + 2 * (sd.tile_off + gb) : a.ext_boxes + 2 * gb;
            blo = bb[0];
            bhi = bb[1];
        }
        const float4 *gh = a.src_hi + sd.src_off;
        const float4 *gl = a.src_lo + sd.src_off;
        const int ntile = t1 - t0;
        auto issue = [&](int k, int buf) {
            long long s0 = (long long)(t0 + k) * TILE;
            int cnt = (int)min((long long)TILE, Ns - s0);
            uint32_t bytes = (uint32_t)cnt * 16u;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[buf], 2u * bytes);
            bulk_g2s(sh_hi + buf * TILE, gh + s0, bytes, &bar[buf]);
            bulk_g2s(sh_lo + buf * TILE, gl + s0, bytes, &bar[buf]);
        };
        if (tid == 0) {
            if (ntile > 0) issue(0, 0);
            if (ntile > 1) issue(1, 1);
        }
        for (int k = 0; k < ntile; ++k) {
            const int buf = k & 1;
            if (!mbar_wait_bounded(&bar[buf], parity[buf])) {
                s_abort = 1;
                atomicOr(&a.status[it.sys], ST_TIMEOUT);
            }
            parity[buf] ^= 1u;
            const long long s0 = (long long)(t0 + k) * TILE;
            const int cnt = (int)min((long long)TILE, Ns - s0);
            constexpr int FOLD = X2 ? kFold2 : kFold;
            const int cnt_pad = (cnt + FOLD - 1) / FOLD * FOLD;
            float4 *bh = sh_hi + buf * TILE;
            float4 *bl = sh_lo + buf * TILE;
            const int skip = part ? ((s0 < tb_hi && s0 + cnt > tb_lo) ? 1 : 0) : (a.ext_skip_zero ? 2 : 0);
            int self_rel[T];
#pragma unroll
            for (int t = 0; t < T; ++t) self_rel[t] = (int)(tidx[t] - s0);
            bool far = false;
            if (use_boxes && skip == 0) {
                const float4 slo = a.boxes[2 * (sd.tile_off + t0 + k)];
                const float4 shi = a.boxes[2 * (sd.tile_off + t0 + k) + 1];
                float gx = fmaxf(0.f, fmaxf(slo.x - bhi.x, blo.x - shi.x));
                float gy = fmaxf(0.f, fmaxf(slo.y - bhi.y, blo.y - shi.y));
                float gz = fmaxf(0.f, fmaxf(slo.z - bhi.z, blo.z - shi.z));
                far = gx * gx + gy * gy + gz * gz >= a.far2;
            }
            if constexpr (MODE == 2) {
                // interleave the staged tile in place (low words only for near
                // tiles); the buffer is refilled once the tile is done
                interleave_pairs(bh, bh, cnt, cnt_pad, make_float4(kFar, -kFar, kFar, 0.f), tid);
                if (!far) interleave_pairs(bl, bl, cnt, cnt_pad, make_float4(0.f, 0.f, 0.f, 0.f), tid);
                fence_proxy_async_smem();  // these writes precede the buffer's next bulk copy
                __syncthreads();
                if (s_abort) break;
                if (field) {
                    if (far)
                        tile32x2<T, UNROLL, true, 0, false, true>(bh, bl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                    else if (skip == 1)
                        tile32x2<T, UNROLL, true, 1, true, true>(bh, bl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                    else if (skip == 2)
                        tile32x2<T, UNROLL, true, 2, true, true>(bh, bl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                    else
                        tile32x2<T, UNROLL, true, 0, true, true>(bh, bl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                } else {
                    if (far)
                        tile32x2<T, UNROLL, false, 0, false, true>(bh, bl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                    else if (skip == 2)
                        tile32x2<T, UNROLL, false, 2, true, true>(bh, bl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                    else
                        tile32x2<T, UNROLL, false, 0, true, true>(bh, bl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                }
                __syncthreads();
                if (tid == 0 && k + 2 < ntile) issue(k + 2, buf);
                continue;
            }
            if constexpr (MODE == 1) {
                // interleave the staged tile (low words only for near tiles),
                // then hand the staging buffer back to the copy engine at once
                float4 *ch = cp_hi + (kCpDouble ? buf * TILE : 0);
                float4 *cl = cp_lo + (kCpDouble ? buf * TILE : 0);
                interleave_pairs(bh, ch, cnt, cnt_pad, make_float4(kFar, -kFar, kFar, 0.f), tid);
                if (!far) interleave_pairs(bl, cl, cnt, cnt_pad, make_float4(0.f, 0.f, 0.f, 0.f), tid);
                __syncthreads();
                if (s_abort) break;
                if (tid == 0 && k + 2 < ntile) issue(k + 2, buf);
                if (field) {
                    if (far)
                        tile32x2<T, UNROLL, true, 0, false, false>(ch, cl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                    else if (skip == 1)
                        tile32x2<T, UNROLL, true, 1, true, false>(ch, cl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                    else if (skip == 2)
                        tile32x2<T, UNROLL, true, 2, true, false>(ch, cl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                    else
                        tile32x2<T, UNROLL, true, 0, true, false>(ch, cl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                } else {
                    if (far)
                        tile32x2<T, UNROLL, false, 0, false, false>(ch, cl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                    else if (skip == 2)
                        tile32x2<T, UNROLL, false, 2, true, false>(ch, cl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                    else
                        tile32x2<T, UNROLL, false, 0, true, false>(ch, cl, cnt_pad, nth, ntl, self_rel, phi, g, acc);
                }
                // one interleaved buffer: it is rewritten next, wait for every
                // warp; two: the barrier after the next interleave suffices
                if (!kCpDouble) __syncthreads();
                continue;
            }
            if (cnt_pad > cnt) {
                for (int s = cnt + tid; s < cnt_pad; s += kThreads) {
                    bh[s] = make_float4(kFar, -kFar, kFar, 0.f);
                    bl[s] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                fence_proxy_async_smem();  // these writes precede the buffer's next bulk copy
            }
            __syncthreads();
            if (s_abort) break;
            if (field) {
                if (far)
                    tile32<T, UNROLL, true, 0, false>(bh, bl, cnt_pad, th, tl, self_rel, phi, g);
                else if (skip == 1)
                    tile32<T, UNROLL, true, 1, true>(bh, bl, cnt_pad, th, tl, self_rel, phi, g);
                else if (skip == 2)
                    tile32<T, UNROLL, true, 2, true>(bh, bl, cnt_pad, th, tl, self_rel, phi, g);
                else
                    tile32<T, UNROLL, true, 0, true>(bh, bl, cnt_pad, th, tl, self_rel, phi, g);
            } else {
                if (far)
                    tile32<T, UNROLL, false, 0, false>(bh, bl, cnt_pad, th, tl, self_rel, phi, g);
                else if (skip == 2)
                    tile32<T, UNROLL, false, 2, true>(bh, bl, cnt_pad, th, tl, self_rel, phi, g);
                else
                    tile32<T, UNROLL, false, 0, true>(bh, bl, cnt_pad, th, tl, self_rel, phi, g);
            }
            __syncthreads();
            if (tid == 0 && k + 2 < ntile) issue(k + 2, buf);
        }
        if (s_abort) {
            // give copies still in flight a bounded chance to land before exit
            for (int b = 0; b < 2; ++b) mbar_wait_bounded(&bar[b], parity[b], 200000000LL);
            break;
        }
        float4 *rec = a.partials + 2 * (sd.partial_off + (long long)it.chunk * ntgt);
        if constexpr (SACC) {
#pragma unroll
            for (int t = 0; t < T; ++t) {
                phi[t] = acc[t * kThreads];
#pragma unroll
                for (int c = 0; c < 3; ++c) g[t][c] = acc[(T + 3 * t + c) * kThreads];
            }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
            if (tidx[t] < 0) continue;
            rec[2 * tidx[t]] = make_float4(phi[t].x, phi[t].y, g[t][0].x, g[t][0].y);
            rec[2 * tidx[t] + 1] = make_float4(g[t][1].x, g[t][1].y, g[t][2].x, g[t][2].y);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ FP64 tiles
template <bool FIELD, int SKIP>
__device__ __forceinline__ void tile64(const double4_32a *__restrict__ s4, int cnt, const double (&tx)[kT64][3],
                                       const int (&self_rel)[kT64], double (&phi)[kT64], double (&g)[kT64][3])
{
#pragma unroll 2
    for (int s = 0; s < cnt; ++s) {
        const double4_32a p = s4[s];
#pragma unroll
        for (int t = 0; t < kT64; ++t) {
            double dx = p.x - tx[t][0];
            double dy = p.y - tx[t][1];
            double dz = p.z - tx[t][2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double ri = rsqrt(r2);
            if (SKIP == 1) ri = (s == self_rel[t]) ? 0.0 : ri;
            if (SKIP == 2) ri = (r2 > 0.0) ? ri : 0.0;
            double qr = p.w * ri;
            phi[t] += qr;
            if (FIELD) {
                double qr3 = qr * ri * ri;
                g[t][0] += qr3 * dx;
                g[t][1] += qr3 * dy;
                g[t][2] += qr3 * dz;
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads, 4) pair_fp64_kernel(PairArgs a)
{
    extern __shared__ __align__(128) double4_32a smem64[];  // [2][kTile64]
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_item, s_abort;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
        s_abort = 0;
    }
    __syncthreads();
    uint32_t parity[2] = {0u, 0u};

    for (int round = 0;; ++round) {
        if (tid == 0) s_item = a.one_item ? (round == 0 ? (int)blockIdx.x : a.total_items) : atomicAdd(a.next_item, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.total_items || s_abort) break;
        const Item it = decode_item(a, item);
        const SysDesc sd = a.sys[it.sys];
        const long long Ns = a.ns[it.sys];
        const long long ntiles = (Ns + kTile64 - 1) / kTile64;
        const int t0 = (int)(it.chunk * ntiles / sd.nchunks);
        const int t1 = (int)((it.chunk + 1) * ntiles / sd.nchunks);
        const bool part = it.tb < sd.ntb_part;
        const bool field = part || a.ext_field;
        const long long ntgt = sd.n + a.n_ext;
        const int gb = part ? sd.pb_lo + it.tb : sd.mb_lo + it.tb - sd.ntb_part;

        double tx[kT64][3];
        long long tidx[kT64];
        long long tb_lo = 0, tb_hi = 0;
        if (part) {
            tb_lo = (long long)gb * kTB64;
            tb_hi = tb_lo + kTB64;
        }
#pragma unroll
        for (int t = 0; t < kT64; ++t) {
            long long k = (long long)gb * kTB64 + t * kThreads + tid;
            bool valid = part ? (k < sd.n) : (k < a.n_ext);
            double4_32a p = make_double4_32a(1e4, 1e4, 1e4, 0.0);
            if (valid) p = part ? a.src64[sd.src_off + k] : a.ext64[k];
            tx[t][0] = p.x; tx[t][1] = p.y; tx[t][2] = p.z;
            tidx[t] = valid ? (part ? k : sd.n + k) : -1;
        }
        double phi[kT64], g[kT64][3];
#pragma unroll
        for (int t = 0; t < kT64; ++t) phi[t] = g[t][0] = g[t][1] = g[t][2] = 0.0;

        const double4_32a *gs = a.src64 + sd.src_off;
        const int ntile = t1 - t0;
        auto issue = [&](int k, int buf) {
            long long s0 = (long long)(t0 + k) * kTile64;
            int cnt = (int)min((long long)kTile64, Ns - s0);
            uint32_t bytes = (uint32_t)cnt * 32u;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[buf], bytes);
            bulk_g2s(smem64 + buf * kTile64, gs + s0, bytes, &bar[buf]);
        };
        if (tid == 0) {
            if (ntile > 0) issue(0, 0);
            if (ntile > 1) issue(1, 1);
        }
        for (int k = 0; k < ntile; ++k) {
            const int buf = k & 1;
            if (!mbar_wait_bounded(&bar[buf], parity[buf])) {
                s_abort = 1;
                atomicOr(&a.status[it.sys], ST_TIMEOUT);
            }
            parity[buf] ^= 1u;
            __syncthreads();
            if (s_abort) break;
            const long long s0 = (long long)(t0 + k) * kTile64;
            const int cnt = (int)min((long long)kTile64, Ns - s0);
            const double4_32a *b4 = smem64 + buf * kTile64;
            const int skip = part ? ((s0 < tb_hi && s0 + cnt > tb_lo) ? 1 : 0) : (a.ext_skip_zero ? 2 : 0);
            int self_rel[kT64];
#pragma unroll
            for (int t = 0; t < kT64; ++t) self_rel[t] = (int)(tidx[t] - s0);
            if (field) {
                if (skip == 1)
                    tile64<true, 1>(b4, cnt, tx, self_rel, phi, g);
                else if (skip == 2)
                    tile64<true, 2>(b4, cnt, tx, self_rel, phi, g);
                else
                    tile64<true, 0>(b4, cnt, tx, self_rel, phi, g);
            } else {
                if (skip == 2)
                    tile64<false, 2>(b4, cnt, tx, self_rel, phi, g);
                else
                    tile64<false, 0>(b4, cnt, tx, self_rel, phi, g);
            }
            __syncthreads();
            if (tid == 0 && k + 2 < ntile) issue(k + 2, buf);
        }
        if (s_abort) {
            for (int b = 0; b < 2; ++b) mbar_wait_bounded(&bar[b], parity[b], 200000000LL);
            break;
        }
        double4_32a *rec = reinterpret_cast<double4_32a *>(a.partials) + (sd.partial_off + (long long)it.chunk * ntgt);
#pragma unroll
        for (int t = 0; t < kT64; ++t) {
            if (tidx[t] < 0) continue;
            rec[tidx[t]] = make_double4_32a(phi[t], g[t][0], g[t][1], g[t][2]);
        }
        __syncthreads();
    }
}

// Sum the chunk partials of every target (deterministic: four running sums
// over the chunks c = 0, 1, 2, 3 mod 4, each in chunk order, then added in a
// fixed order; the four independent streams keep four loads per thread in
// flight).  FP32 records are double-float values and are summed in
// double-float arithmetic on the FP32 pipe (FP64 issue is far slower on this
// part); the total is converted to FP64 once.
// phi_tgt[tgt_off + t] = potential, e_part[3 (tgt_off + t) + a] = field
// E = -sum q (y - x)/r^3.
__global__ void partial_reduce_kernel(const SysDesc *sys, int n_ext, const float4 *partials, int precision,
                                      double *phi_tgt, double *e_part)
{
    const SysDesc sd = sys[blockIdx.y];
    long long ntgt = sd.n + n_ext;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntgt) return;
    const int nc = sd.nchunks;
    const long long o = sd.tgt_off + t;
    if (precision == HSMA_FP64) {
        double p[4] = {0.0, 0.0, 0.0, 0.0}, gx[4] = {0.0, 0.0, 0.0, 0.0}, gy[4] = {0.0, 0.0, 0.0, 0.0},
               gz[4] = {0.0, 0.0, 0.0, 0.0};
        const double4_32a *rec = reinterpret_cast<const double4_32a *>(partials) + sd.partial_off + t;
        int c = 0;
        for (; c + 4 <= nc; c += 4) {
            double4_32a r[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) r[j] = rec[(long long)(c + j) * ntgt];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                p[j] += r[j].x;
                gx[j] += r[j].y;
                gy[j] += r[j].z;
                gz[j] += r[j].w;
            }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (c + j >= nc) break;
            double4_32a r = rec[(long long)(c + j) * ntgt];
            p[j] += r.x;
            gx[j] += r.y;
            gy[j] += r.z;
            gz[j] += r.w;
        }
        phi_tgt[o] = (p[0] + p[1]) + (p[2] + p[3]);
        e_part[3 * o] = -((gx[0] + gx[1]) + (gx[2] + gx[3]));
        e_part[3 * o + 1] = -((gy[0] + gy[1]) + (gy[2] + gy[3]));
        e_part[3 * o + 2] = -((gz[0] + gz[1]) + (gz[2] + gz[3]));
        return;
    }
    const float2 z2 = make_float2(0.f, 0.f);
    float2 p[4] = {z2, z2, z2, z2}, gx[4] = {z2, z2, z2, z2}, gy[4] = {z2, z2, z2, z2}, gz[4] = {z2, z2, z2, z2};
    const float4 *rec = partials + 2 * (sd.partial_off + t);
    int c = 0;
    for (; c + 4 <= nc; c += 4) {
        float4 r0[4], r1[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            r0[j] = rec[2 * (long long)(c + j) * ntgt];
            r1[j] = rec[2 * (long long)(c + j) * ntgt + 1];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            p[j] = df_add_df(p[j], make_float2(r0[j].x, r0[j].y));
            gx[j] = df_add_df(gx[j], make_float2(r0[j].z, r0[j].w));
            gy[j] = df_add_df(gy[j], make_float2(r1[j].x, r1[j].y));
            gz[j] = df_add_df(gz[j], make_float2(r1[j].z, r1[j].w));
        }
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (c + j >= nc) break;
        const float4 r0 = rec[2 * (long long)(c + j) * ntgt];
        const float4 r1 = rec[2 * (long long)(c + j) * ntgt + 1];
        p[j] = df_add_df(p[j], make_float2(r0.x, r0.y));
        gx[j] = df_add_df(gx[j], make_float2(r0.z, r0.w));
        gy[j] = df_add_df(gy[j], make_float2(r1.x, r1.y));
        gz[j] = df_add_df(gz[j], make_float2(r1.z, r1.w));
    }
    auto total = [](const float2 (&v)[4]) {
        const float2 s = df_add_df(df_add_df(v[0], v[1]), df_add_df(v[2], v[3]));
        return (double)s.x + (double)s.y;
    };
    phi_tgt[o] = total(p);
    e_part[3 * o] = -total(gx);
    e_part[3 * o + 1] = -total(gy);
    e_part[3 * o + 2] = -total(gz);
}

}  // namespace

// FP32 kernel variants (the autotuner's candidates):
//   4 = four targets per thread, scalar loop, >= 4 CTAs/SM
//   5 = four targets, scalar, >= 5 CTAs/SM
//   2 = two targets, scalar, >= 6 CTAs/SM
//  12 = two targets, packed two-source loop (mode 1), >= 6 CTAs/SM
//  13 = two targets, packed (mode 1), >= 5 CTAs/SM
//  14 = four targets, packed (mode 1), >= 3 CTAs/SM
//  15 = four targets, packed in place, shared accumulators (mode 2), >= 4 CTAs/SM
//  16 = two targets, packed in place, shared accumulators (mode 2), >= 6 CTAs/SM
//  17 = three targets (blocks and tiles of 384), packed (mode 1), >= 4 CTAs/SM
bool pair_variant_valid(int variant)
{
    switch (variant) {
    case 2: case 4: case 5: case 12: case 13: case 14: case 15: case 16: case 17: return true;
    default: return false;
    }
}

static int variant_targets(int variant)
{
    if (variant == 17) return 3;
    return (variant == 2 || variant == 12 || variant == 13 || variant == 16) ? 2 : 4;
}
static int variant_mode(int variant) { return variant == 17 ? 1 : (variant >= 15 ? 2 : (variant >= 12 ? 1 : 0)); }

int pair_targets_per_block(int precision, int variant)
{
    return precision == HSMA_FP64 ? kTB64 : kThreads * variant_targets(variant);
}

static size_t pair_smem(int precision, int variant)
{
    if (precision == HSMA_FP64) return 2 * kTile64 * sizeof(double4_32a);
    // staging: 2 buffers x (hi, lo); mode 1 adds the interleaved (hi, lo),
    // mode 2 the 4T double-float accumulators of every thread
    const size_t tile = (size_t)pair_targets_per_block(precision, variant);
    const int mode = variant_mode(variant);
    const size_t extra = mode == 1 ? (kCpDouble ? 4 : 2) * tile * sizeof(float4)
                                   : (mode == 2 ? 4 * (size_t)variant_targets(variant) * kThreads * sizeof(float2) : 0);
    return 4 * tile * sizeof(float4) + extra;
}

template <class K>
static int occupancy_of(K kernel, size_t sm)
{
    int n = 0;
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kThreads, sm);
    return n > 0 ? n : 1;
}

int pair_max_ctas_per_sm(int precision, int variant)
{
    const size_t sm = pair_smem(precision, variant);
    if (precision == HSMA_FP64) return occupancy_of(pair_fp64_kernel, sm);
    switch (variant) {
    case 2: return occupancy_of(pair_fp32_kernel<2, 6, 0>, sm);
    case 5: return occupancy_of(pair_fp32_kernel<4, 5, 0>, sm);
    case 12: return occupancy_of(pair_fp32_kernel<2, 6, 1>, sm);
    case 13: return occupancy_of(pair_fp32_kernel<2, 5, 1>, sm);
    case 14: return occupancy_of(pair_fp32_kernel<4, 3, 1>, sm);
    case 15: return occupancy_of(pair_fp32_kernel<4, 4, 2>, sm);
    case 16: return occupancy_of(pair_fp32_kernel<2, 6, 2>, sm);
    case 17: return occupancy_of(pair_fp32_kernel<3, 4, 1>, sm);
    default: return occupancy_of(pair_fp32_kernel<4, 4, 0>, sm);
    }
}

// The dynamic shared-memory attribute is set by pair_max_ctas_per_sm, which
// every caller runs before its first launch (so that launches can be
// captured into a CUDA graph).
int launch_pair(const PairArgs &a, int precision, int variant, int grid, cudaStream_t st)
{
    if (a.total_items <= 0) return HSMA_OK;
    const size_t sm = pair_smem(precision, variant);
    if (precision == HSMA_FP64) {
        pair_fp64_kernel<<<grid, kThreads, sm, st>>>(a);
    } else {
        switch (variant) {
        case 2: pair_fp32_kernel<2, 6, 0><<<grid, kThreads, sm, st>>>(a); break;
        case 5: pair_fp32_kernel<4, 5, 0><<<grid, kThreads, sm, st>>>(a); break;
        case 12: pair_fp32_kernel<2, 6, 1><<<grid, kThreads, sm, st>>>(a); break;
        case 13: pair_fp32_kernel<2, 5, 1><<<grid, kThreads, sm, st>>>(a); break;
        case 14: pair_fp32_kernel<4, 3, 1><<<grid, kThreads, sm, st>>>(a); break;
        case 15: pair_fp32_kernel<4, 4, 2><<<grid, kThreads, sm, st>>>(a); break;
        case 16: pair_fp32_kernel<2, 6, 2><<<grid, kThreads, sm, st>>>(a); break;
        case 17: pair_fp32_kernel<3, 4, 1><<<grid, kThreads, sm, st>>>(a); break;
        default: pair_fp32_kernel<4, 4, 0><<<grid, kThreads, sm, st>>>(a); break;
        }
    }
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

int launch_partial_reduce(const SysDesc *sys, int nsys, long long max_tgt, int n_ext, const float4 *partials,
                          int precision, double *phi_tgt, double *e_part, cudaStream_t st)
{
    dim3 grid((unsigned)((max_tgt + 255) / 256), nsys);
    partial_reduce_kernel<<<grid, 256, 0, st>>>(sys, n_ext, partials, precision, phi_tgt, e_part);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    return HSMA_OK;
}

}  // namespace hsma
