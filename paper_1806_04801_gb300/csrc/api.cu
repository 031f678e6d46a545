// C ABI of libhsma (declared in include/hsma.h): plan construction
// (preparation step, Sec. II.C) and the update step orchestration.  All
// arithmetic of the method runs in the kernels of the other translation
// units; this file validates arguments, lays out device memory and enqueues
// work on the plan's stream.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace hsma {

std::atomic<long long> g_launches{0};
std::atomic<long long> g_alloc_calls{0};
static thread_local char g_cuda_err[384];

void set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s (%s) at %s:%d: %s", cudaGetErrorName(e), what, file, line,
             cudaGetErrorString(e));
}

int surface_targets_per_block();

}  // namespace hsma

using namespace hsma;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kInsetBlock = 256;
// Size limits of the update step.  Systems and image shifts index grid
// dimensions y / z of several kernels (at most 65535 each; the tensor-core
// fit pads the system count to a multiple of 8, hence 65528); a system's
// in-set slots, particle indices and work items are 32-bit.
constexpr int kMaxSystems = 65528;
constexpr int kMaxShifts = 65535;
constexpr long long kMaxInsetSlots = (1LL << 31) - 1;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Bump allocator over one device allocation.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base((char *)b) {}
    template <class T>
    T *take(size_t count)
    {
        off = align_up(off, 256);
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

struct Workspace {
    double *xyz = nullptr, *q = nullptr;            // staged inputs (host-input calls)
    double *forces = nullptr, *pot = nullptr;       // staged outputs (host-output calls)
    float4 *src_hi = nullptr, *src_lo = nullptr;    // in-set, FP32 split form
    double4_32a *src64 = nullptr;                       // in-set, FP64
    int *counts = nullptr;
    long long *ns = nullptr;
    int *keys = nullptr, *perm = nullptr, *keys2 = nullptr, *vals2 = nullptr, *hist = nullptr;
    float4 *boxes = nullptr;
    float4 *partials = nullptr;
    double *phi_tgt = nullptr, *e_part = nullptr;
    double *b = nullptr, *A = nullptr;
    double2 *img = nullptr;
    double *phi_out = nullptr, *e_out = nullptr;
    double *energy = nullptr, *upart = nullptr;
    int *status = nullptr;
    int *ctrl = nullptr;                            // work counters
    SysDesc *sys = nullptr;
    float *tc_work = nullptr;
    long long *idx64 = nullptr;                     // target sharding: caller indices of a slice
    double4_32a *cen = nullptr;                     // in-set scratch: centred particles, spatial order
    float4 *cenf = nullptr;                         // the same in FP32
    double2 *qsums = nullptr;                       // per particle block: (sum q, sum |q|)
};

struct BatchShape {
    int nsys = 0;
    long long n_total = 0, cap_total = 0, cnt_total = 0, rec_total = 0, tgt_total = 0, hist_total = 0,
              tiles_total = 0, max_tiles = 0;
    int items = 0, surf_items = 0, nblk_max = 1;
    long long max_tgt = 0, max_n = 0;
    int variant = 4;
    std::vector<SysDesc> sys;
};

}  // namespace

struct hsma_plan_s {
    double L[3];
    int bc, P, Nb, ncols, K, nmon, F2, F1, ndir, nshifts;
    double Rs, R0, dr, alpha, cond;
    double far_rel = 1.0 / 15.0;  // near/far threshold of the FP32 pair sums, in units of Rs
    int stall_test = 0;           // HSMA_TEST_STALL_WAIT=1 at plan creation: exercise the timeout path
    int preemptible = 0;          // pair work as one CTA per item (see hsma_plan_set_preemptible)
    int far_field = 0;            // 0: surface images (Sec. II.B); 1: direct series at the particles
    int precision, use_graphs, profile, mon_faces;
    cudaStream_t stream;
    int num_sms, ctas[3];
    static constexpr int kVariantCodes = 32;
    int ctas_var[kVariantCodes] = {};  // FP32 pair kernel: resident CTAs per SM, by variant code
    // tuning of the pair kernel: a fixed choice, or entries per work bucket
    bool tune_fixed = false;
    hsma_tuning tune_value{4, 24, 0.0};
    std::vector<std::pair<int, hsma_tuning>> tune_entries;  // (bucket, tuning)
    char device_name[256] = {0};
    // plan-resident device data
    void *plan_mem = nullptr;
    double4_32a *mon64 = nullptr;
    float4 *mon_hi = nullptr, *mon_lo = nullptr;
    // monitoring targets in spatial (Morton) order for the pair kernel
    double4_32a *mon64_s = nullptr;
    float4 *mon_hi_s = nullptr, *mon_lo_s = nullptr, *mon_boxes = nullptr, *mon_boxes2 = nullptr;
    float4 *mon_boxes3 = nullptr;  // monitoring-target block boxes for blocks of 512 / 256 / 384
    int *mon_perm_d = nullptr, *mon_inv = nullptr;
    std::vector<int> mon_perm;
    double *Mrow = nullptr, *Mp = nullptr, *Bq = nullptr, *norm = nullptr;
    double4_32a *dirs = nullptr;
    int4 *shifts = nullptr;
    void *tc_hi = nullptr, *tc_lo = nullptr;
    void *tc_mdf = nullptr;  // M (K x n_cols) as FP32 word pairs, for the refinement residual
    // workspace
    void *ws_mem = nullptr;
    size_t ws_cap = 0;
    Workspace ws;
    // pinned host staging
    void *hpin = nullptr;
    size_t hpin_cap = 0;
    // last call
    int last_nsys = 0;
    long long last_n = 0;
    BatchShape last_shape;
    cudaEvent_t ev[8] = {};
    bool events_ready = false;
    double last_ms[8] = {};
    bool have_timings = false;
    // CUDA graphs of the update step: the last few batch shapes / step modes
    struct GraphEntry {
        std::vector<long long> key;
        cudaGraphExec_t exec = nullptr;
        long long kernels = 0;
        long long last_use = 0;
    };
    std::vector<GraphEntry> graphs;
    long long graph_clock = 0;
    // reusable in-set for repeated single-system steps (molecular dynamics):
    // a candidate list at Rs + skin over an enlarged shift table, the Morton
    // order and the centred positions of its build
    double md_skin = 0.0;
    bool md_valid = false;
    long long md_n = 0, md_ncand = 0;
    int md_prec = -1, md_nshifts = 0;
    std::vector<int4> md_shift_host;
    void *md_mem = nullptr;
    size_t md_cap = 0;
    int2 *md_cand = nullptr;
    int *md_perm = nullptr, *md_counts = nullptr, *md_rcounts = nullptr;
    double4_32a *md_x0 = nullptr, *md_u = nullptr;
    int4 *md_shifts = nullptr;
    long long *md_ns = nullptr, *md_ns_host = nullptr;
    bool md_shifts_dirty = true;
    long long md_builds = 0, md_reuses = 0, md_stale = 0;
    cudaStream_t priv_stream = nullptr;
    cudaEvent_t order_ev = nullptr;
};

namespace {

std::vector<long long> fibonacci_list()
{
    std::vector<long long> f = {1, 2};
    while (f.back() < 100000000LL) f.push_back(f[f.size() - 1] + f[f.size() - 2]);
    return f;
}

// F2 such that 6(F2+1) is nearest to Q (ties to the larger F2); F1 its predecessor.
void fib_from_q(int Q, int *F2, int *F1)
{
    auto f = fibonacci_list();
    long long bestd = -1;
    for (size_t i = 1; i < f.size(); ++i) {
        long long d = llabs(6 * (f[i] + 1) - Q);
        if (bestd < 0 || d < bestd || (d == bestd && f[i] > *F2)) {
            bestd = d;
            *F2 = (int)f[i];
            *F1 = (int)f[i - 1];
        }
    }
}

bool fib_pred(int F2, int *F1)
{
    auto f = fibonacci_list();
    for (size_t i = 1; i < f.size(); ++i)
        if (f[i] == F2) {
            *F1 = (int)f[i - 1];
            return true;
        }
    return false;
}

// Image shells per axis: the smallest k with (k + 1/2) L_a >= Rs.  A sphere
// 1e5 box lengths across or more returns 1e5, far beyond any shift table.
int shells(double Rs, double La)
{
    if (!(Rs / La < 1e5)) return 100000;
    int k = 0;
    while ((k + 1) * La - 0.5 * La < Rs) ++k;
    return k;
}

int map_status(int st)
{
    if (st & ST_OUT_OF_BOX) return HSMA_E_OUT_OF_BOX;
    if (st & ST_NONNEUTRAL) return HSMA_E_NONNEUTRAL;
    if (st & ST_TIMEOUT) return HSMA_E_TIMEOUT;
    if (st & ST_CAPACITY) return HSMA_E_ARG;
    if (st & ST_COINCIDENT) return HSMA_E_COINCIDENT;
    return HSMA_OK;
}

int ensure_pinned(hsma_plan_s *p, size_t bytes)
{
    if (bytes <= p->hpin_cap) return HSMA_OK;
    if (p->hpin) host_free(p->hpin);
    p->hpin = nullptr;
    p->hpin_cap = 0;
    size_t nb = std::max(bytes, (size_t)65536);
    HSMA_CUDA_TRY(host_malloc(&p->hpin, nb));
    p->hpin_cap = nb;
    return HSMA_OK;
}

// CTAs of the cooperative tensor-core fit: one per SM, or a quarter of the
// SMs for a preemptible plan (a cooperative launch needs all its CTAs
// resident at once, which a smaller grid finds sooner beside other work).
int fit_ctas(const hsma_plan_s *p) { return p->preemptible ? std::max(8, p->num_sms / 4) : p->num_sms; }

constexpr int kPreemptibleItemsFactor = 8;  // work items of a preemptible plan per tuned item

// Work decomposition of a batch: targets per block, source chunks per system,
// work items, surface blocks.  Pure host arithmetic.
int tuned_ctas(const hsma_plan_s *p, int precision, int variant)
{
    if (precision == HSMA_FP64) return p->ctas[0];
    return (variant > 0 && variant < hsma_plan_s::kVariantCodes && p->ctas_var[variant] > 0) ? p->ctas_var[variant]
                                                                                             : p->ctas[1];
}

// Pair work of a batch (targets x estimated in-set sources), and its bucket
// (floor of log2) that keys the tuning entries.
double batch_work(const hsma_plan_s *p, int nsys, const long long *n)
{
    const double vsphere = 4.0 / 3.0 * kPi * p->Rs * p->Rs * p->Rs;
    const double vbox = p->L[0] * p->L[1] * p->L[2];
    double w = 0.0;
    for (int s = 0; s < nsys; ++s)
        w += (double)(n[s] + p->nmon) * std::min((double)n[s] * p->nshifts, (double)n[s] * vsphere / vbox);
    return w;
}

int work_bucket(double w) { return w > 1.0 ? (int)floor(log2(w)) : 0; }

hsma_tuning choose_tuning(const hsma_plan_s *p, int nsys, const long long *n)
{
    if (p->tune_fixed) return p->tune_value;
    const int b = work_bucket(batch_work(p, nsys, n));
    const hsma_tuning *best = nullptr;
    int bestd = 1 << 30;
    for (auto &e : p->tune_entries) {
        int d = abs(e.first - b);
        if (d < bestd && d <= 1) {
            bestd = d;
            best = &e.second;
        }
    }
    if (best) return *best;
    // untuned: the packed variants measured fastest on this part, four targets
    // per thread for one system, three for a batch
    return p->precision == HSMA_FP64 ? hsma_tuning{4, 24, 0.0} : hsma_tuning{nsys > 1 ? 17 : 14, 48, 0.0};
}

void shape_batch(const hsma_plan_s *p, int nsys, const long long *n, int precision, const hsma_tuning &tu,
                 BatchShape *sh)
{
    sh->nsys = nsys;
    sh->sys.assign(nsys, SysDesc{});
    sh->variant = pair_variant_valid(tu.pair_variant) ? tu.pair_variant : 4;
    const int TB = pair_targets_per_block(precision, sh->variant);
    const int STB = surface_targets_per_block();
    const int tile = TB;
    const double vsphere = 4.0 / 3.0 * kPi * p->Rs * p->Rs * p->Rs;
    const double vbox = p->L[0] * p->L[1] * p->L[2];
    const int slots = p->num_sms * tuned_ctas(p, precision, sh->variant);
    const int ntb_mon = (p->nmon + TB - 1) / TB;
    double work = 0.0;
    std::vector<double> ns_est(nsys);
    for (int s = 0; s < nsys; ++s) {
        ns_est[s] = std::max(1.0, std::min((double)n[s] * p->nshifts, (double)n[s] * vsphere / vbox));
        int ntb = (int)((n[s] + TB - 1) / TB) + ntb_mon;
        work += (double)ntb * ns_est[s];
    }
    // preemptible plans cut their items finer, so that an SM frees up (for a
    // higher-priority stream) after a shorter wait
    const double items_wanted =
        (double)std::max(1, tu.items_per_slot) * slots * (p->preemptible ? kPreemptibleItemsFactor : 1);
    // smallest chunk: four tiles (each item re-reads its targets and writes a
    // partial record per target, which the chunk reduction reads back), less --
    // down to one tile -- where four would give fewer than two items per CTA
    // slot (small systems; measured at N = 1000 / 2000: 0.293 -> 0.242 and
    // 0.315 -> 0.290 ms per step, N >= 1e4 unchanged)
    const double chunk =
        std::max(std::min(4.0 * tile, std::max(1.0 * tile, work / (2.0 * slots))), work / items_wanted);
    long long part = 0, src = 0, tgt = 0, rec = 0, cnt = 0, hist = 0, tiles = 0, max_tiles = 0;
    long long items = 0, surf = 0;
    int nblk_max = 1;
    long long max_tgt = 0;
    for (int s = 0; s < nsys; ++s) {
        SysDesc &d = sh->sys[s];
        d.n = n[s];
        d.part_off = part;
        d.src_off = src;
        d.tgt_off = tgt;
        d.nblk = (int)((n[s] + kInsetBlock - 1) / kInsetBlock);
        d.cnt_off = cnt;
        d.hist_off = hist;
        d.tile_off = tiles;
        // Morton grid: about 4 particles per cell, at most 32 cells per axis
        int gb = 1;
        while (gb < 5 && (double)(1 << (3 * gb)) * 4.0 < (double)n[s]) ++gb;
        d.gbits = gb;
        long long tcap = (n[s] * p->nshifts + 255) / 256;  // tiles of the smallest variant
        d.ntb_part = (int)((n[s] + TB - 1) / TB);
        d.ntb = d.ntb_part + ntb_mon;
        long long maxchunks = std::max(1LL, (long long)(ns_est[s] / tile));
        d.nchunks = (int)std::max(1LL, std::min(maxchunks, (long long)llround(ns_est[s] / chunk)));
        d.partial_off = rec;
        d.item_off = (int)items;
        d.surf_off = (int)surf;
        d.sp_lo = 0;
        d.sp_n = n[s];
        d.pb_lo = 0;
        d.mb_lo = 0;
        long long ntgt = n[s] + p->nmon;
        part += n[s];
        src += n[s] * p->nshifts;
        tgt += ntgt;
        rec += (long long)d.nchunks * ntgt;
        cnt += (long long)p->nshifts * d.nblk;
        hist += 256LL * d.nblk;
        tiles += tcap;
        max_tiles = std::max(max_tiles, tcap);
        items += (long long)d.ntb * d.nchunks;
        surf += (n[s] + STB - 1) / STB;
        nblk_max = std::max(nblk_max, d.nblk);
        max_tgt = std::max(max_tgt, ntgt);
        sh->max_n = std::max(sh->max_n, (long long)n[s]);
    }
    sh->n_total = part;
    sh->cap_total = src;
    sh->tgt_total = tgt;
    sh->rec_total = rec;
    sh->cnt_total = cnt;
    sh->hist_total = hist;
    sh->tiles_total = tiles;
    sh->max_tiles = max_tiles;
    sh->items = items > INT32_MAX ? -1 : (int)items;
    sh->surf_items = surf > INT32_MAX ? -1 : (int)surf;
    sh->nblk_max = nblk_max;
    sh->max_tgt = max_tgt;
}

// Carve the workspace; with base == nullptr only computes the size.
size_t carve_workspace(const hsma_plan_s *p, const BatchShape &sh, int precision, bool stage_in, bool stage_out,
                       void *base, Workspace *w)
{
    Carver c(base);
    w->xyz = stage_in ? c.take<double>(3 * sh.n_total) : nullptr;
    w->q = stage_in ? c.take<double>(sh.n_total) : nullptr;
    w->forces = stage_out ? c.take<double>(3 * sh.n_total) : nullptr;
    w->pot = stage_out ? c.take<double>(sh.n_total) : nullptr;
    if (precision == HSMA_FP64) {
        w->src64 = c.take<double4_32a>(sh.cap_total);
        w->src_hi = w->src_lo = nullptr;
    } else {
        w->src_hi = c.take<float4>(sh.cap_total);
        w->src_lo = c.take<float4>(sh.cap_total);
        w->src64 = nullptr;
    }
    w->counts = c.take<int>(sh.cnt_total);
    w->ns = c.take<long long>(sh.nsys);
    w->keys = c.take<int>(sh.n_total);
    w->perm = c.take<int>(sh.n_total);
    w->keys2 = c.take<int>(sh.n_total);
    w->vals2 = c.take<int>(sh.n_total);
    w->hist = c.take<int>(sh.hist_total);
    w->boxes = (precision == HSMA_FP64) ? nullptr : c.take<float4>(2 * sh.tiles_total);
    w->partials = c.take<float4>(2 * sh.rec_total);
    w->phi_tgt = c.take<double>(sh.tgt_total);
    w->e_part = c.take<double>(3 * sh.tgt_total);
    w->b = c.take<double>((size_t)sh.nsys * p->K);
    w->A = c.take<double>((size_t)sh.nsys * p->Nb);
    w->img = c.take<double2>((size_t)sh.nsys * p->ndir);
    w->phi_out = c.take<double>(sh.n_total);
    w->e_out = c.take<double>(3 * sh.n_total);
    w->energy = c.take<double>(sh.nsys);
    w->upart = c.take<double>((size_t)sh.nsys * finalize_blocks(sh.max_n));
    w->status = c.take<int>(sh.nsys);
    w->ctrl = c.take<int>(8);
    w->sys = c.take<SysDesc>(sh.nsys);
    w->tc_work = (precision == HSMA_FP32_TC_FIT) ? (float *)c.take<char>(tc_work_bytes(p->K, p->ncols, sh.nsys, fit_ctas(p)))
                                                  : nullptr;
    w->idx64 = c.take<long long>(sh.n_total);
    w->cen = c.take<double4_32a>(sh.n_total);
    w->cenf = c.take<float4>(sh.n_total);
    w->qsums = c.take<double2>(sh.cnt_total / std::max(1, p->nshifts) + 1);
    return align_up(c.off, 256);
}

int ensure_workspace(hsma_plan_s *p, size_t bytes)
{
    if (bytes <= p->ws_cap) return HSMA_OK;
    if (p->ws_mem) {
        HSMA_CUDA_TRY(cudaStreamSynchronize(p->stream));
        dev_free(p->ws_mem);
    }
    p->ws_mem = nullptr;
    p->ws_cap = 0;
    size_t nb = align_up(bytes + bytes / 8, 1 << 20);
    cudaError_t e = dev_malloc(&p->ws_mem, nb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = dev_malloc(&p->ws_mem, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p->ws_mem = nullptr;
            return HSMA_E_OOM;
        }
        nb = bytes;
    }
    p->ws_cap = nb;
    return HSMA_OK;
}

std::vector<double> norm_table(int P)
{
    std::vector<double> v((P + 1) * (P + 1));
    for (int n = 0; n <= P; ++n)
        for (int m = -n; m <= n; ++m) v[n * n + n + m] = basis_norm(n, abs(m));
    return v;
}

void drop_graphs(hsma_plan_s *p)
{
    for (auto &e : p->graphs) cudaGraphExecDestroy(e.exec);
    p->graphs.clear();
}

void record(hsma_plan_s *p, cudaStream_t st, int i)
{
    if (p->profile && p->events_ready) cudaEventRecord(p->ev[i], st);
}

// Every kernel of the update step, enqueued on `st`.  Reads its inputs from
// the workspace staging buffers and writes forces/potentials to the staging
// outputs, so the same sequence can be captured once into a CUDA graph and
// replayed for every call with the same batch shape.
// Step modes for repeated single-system calls (in-set reuse, see
// hsma_plan_set_inset_skin): kFull builds the in-set from scratch; kBuild
// does the same and also records the candidate list, Morton order and
// positions; kReuse regenerates the in-set from the list instead of sorting
// and building.
enum StepMode { kFull = 0, kBuild = 1, kReuse = 2 };

int enqueue_update(hsma_plan_s *p, const BatchShape &sh, const Workspace &w, int prec, bool want_f, bool want_p,
                   int mode, cudaStream_t st)
{
    const int nsys = sh.nsys;
    int rc = HSMA_OK;
    HSMA_CUDA_TRY(cudaMemsetAsync(w.status, 0, sizeof(int) * nsys, st));
    HSMA_CUDA_TRY(cudaMemsetAsync(w.ctrl, 0, sizeof(int) * 8, st));
    record(p, st, 0);
    const int *perm = w.perm;
    if (mode == kReuse) {
        RegenArgs r;
        r.n = sh.sys[0].n;
        r.cap = sh.cap_total;
        r.cap_cand = r.n * p->md_nshifts;
        r.counts = p->md_rcounts;
        r.u = p->md_u;
        r.ncand = p->md_ns;
        r.cand = p->md_cand;
        r.shifts = p->md_shifts;
        r.perm = p->md_perm;
        r.x0 = p->md_x0;
        r.xyz = w.xyz;
        r.q = w.q;
        for (int a = 0; a < 3; ++a) r.g.L[a] = p->L[a];
        r.g.Rs = p->Rs;
        r.g.bc = p->bc;
        r.skin = p->md_skin;
        r.src_hi = w.src_hi;
        r.src_lo = w.src_lo;
        r.src64 = w.src64;
        r.ns = w.ns;
        r.status = w.status;
        if ((rc = launch_inset_regen(r, st))) return rc;
        perm = p->md_perm;
    } else {

    // spatial order of the particles (Morton, stable radix sort)
    SortArgs sa;
    sa.sys = w.sys;
    sa.nsys = nsys;
    sa.xyz = w.xyz;
    for (int a = 0; a < 3; ++a) sa.g.L[a] = p->L[a];
    sa.g.Rs = p->Rs;
    sa.g.bc = p->bc;
    sa.keys = w.keys;
    sa.vals = w.perm;
    sa.keys2 = w.keys2;
    sa.vals2 = w.vals2;
    sa.hist = w.hist;
    if ((rc = launch_sort_particles(sa, sh.nblk_max, st))) return rc;

    // (a1) in-set
    InsetArgs ia;
    ia.sys = w.sys;
    ia.nsys = nsys;
    ia.nblk_max = sh.nblk_max;
    ia.xyz = w.xyz;
    ia.q = w.q;
    ia.perm = w.perm;
    ia.shifts = p->shifts;
    ia.n_shifts = p->nshifts;
    for (int a = 0; a < 3; ++a) ia.g.L[a] = p->L[a];
    ia.g.Rs = p->Rs;
    ia.g.bc = p->bc;
    ia.counts = w.counts;
    ia.ns = w.ns;
    ia.src_hi = w.src_hi;
    ia.src_lo = w.src_lo;
    ia.src64 = w.src64;
    ia.status = w.status;
    ia.cen = w.cen;
    ia.cenf = w.cenf;
    ia.qsums = w.qsums;
    if ((rc = launch_inset(ia, st))) return rc;
    if (mode == kBuild) {
        // candidates within Rs + skin over the enlarged shift table, and the
        // order and positions they refer to
        InsetArgs ca = ia;
        ca.g.Rs = p->Rs + p->md_skin;
        ca.shifts = p->md_shifts;
        ca.n_shifts = p->md_nshifts;
        ca.counts = p->md_counts;
        ca.ns = p->md_ns;
        ca.src_hi = ca.src_lo = nullptr;
        ca.src64 = nullptr;
        ca.cand = p->md_cand;
        if ((rc = launch_inset_candidates(ca, st))) return rc;
        const long long n0 = sh.sys[0].n;
        HSMA_CUDA_TRY(cudaMemcpyAsync(p->md_perm, w.perm, sizeof(int) * n0, cudaMemcpyDeviceToDevice, st));
        HSMA_CUDA_TRY(cudaMemcpyAsync(p->md_x0, w.cen, sizeof(double4_32a) * n0, cudaMemcpyDeviceToDevice, st));
    }
    }
    const int TB = pair_targets_per_block(prec, sh.variant);
    if (w.boxes && (rc = launch_tile_boxes(w.sys, nsys, sh.max_tiles, w.ns, w.src_hi, TB, w.boxes, st))) return rc;
    record(p, st, 1);

    // (a2) near-field sums at particles and monitoring targets
    PairArgs pa;
    pa.sys = w.sys;
    pa.nsys = nsys;
    pa.total_items = sh.items;
    pa.ns = w.ns;
    pa.src_hi = w.src_hi;
    pa.src_lo = w.src_lo;
    pa.src64 = w.src64;
    pa.ext_hi = p->mon_hi_s;
    pa.ext_lo = p->mon_lo_s;
    pa.ext64 = p->mon64_s;
    pa.n_ext = p->nmon;
    pa.ext_field = 0;
    pa.ext_skip_zero = 0;
    pa.boxes = w.boxes;
    pa.ext_boxes = w.boxes ? (TB == 256 ? p->mon_boxes2 : (TB == 384 ? p->mon_boxes3 : p->mon_boxes)) : nullptr;
    pa.stall_test = p->stall_test;
    pa.far2 = (float)(p->far_rel * p->Rs * p->far_rel * p->Rs);
    pa.partials = w.partials;
    pa.next_item = w.ctrl;
    pa.status = w.status;
    const int ctas = tuned_ctas(p, prec, sh.variant);
    pa.one_item = p->preemptible ? 1 : 0;
    const int grid = p->preemptible ? std::max(1, sh.items) : std::max(1, std::min(sh.items, p->num_sms * ctas));
    if ((rc = launch_pair(pa, prec, sh.variant, grid, st))) return rc;
    record(p, st, 2);
    if ((rc = launch_partial_reduce(w.sys, nsys, sh.max_tgt, p->nmon, w.partials, prec, w.phi_tgt, w.e_part, st)))
        return rc;
    record(p, st, 3);

    // (c) fit
    if (prec == HSMA_FP32_TC_FIT)
        rc = launch_fit_tc(w.sys, nsys, p->bc, p->K, p->ncols, p->Nb, p->tc_hi, p->tc_lo, p->tc_mdf, w.phi_tgt,
                           p->mon_inv, w.b, w.A, w.tc_work, w.status, fit_ctas(p), st);
    else
        rc = launch_fit_fp64(w.sys, nsys, p->bc, p->K, p->ncols, p->Nb, p->Mp, w.phi_tgt, p->mon_inv, w.b, w.A,
                             st);
    if (rc) return rc;
    record(p, st, 4);

    if (p->far_field == 1) {
        // far field by the fitted series evaluated at each particle
        record(p, st, 5);
        if ((rc = launch_series_field(w.sys, nsys, sh.max_n, p->P, p->Rs, p->norm, w.A, w.src_hi, w.src_lo, w.src64,
                                      w.phi_out, w.e_out, st)))
            return rc;
        record(p, st, 6);
    } else {
        // (d) surface images and their sums at the particles
        if ((rc = launch_surface_charges(nsys, p->ndir, p->Nb, p->Bq, p->dirs, w.A, p->Rs, w.img, st))) return rc;
        record(p, st, 5);
        if ((rc = launch_surface_pairs(w.sys, nsys, sh.surf_items, w.ns, w.src_hi, w.src_lo, w.src64, p->ndir,
                                       p->dirs, w.img, p->Rs, p->dr, prec, w.phi_out, w.e_out, st)))
            return rc;
        record(p, st, 6);
    }
    if ((rc = launch_finalize(w.sys, nsys, sh.max_n, perm, w.q, w.phi_tgt, w.e_part, w.phi_out, w.e_out,
                              want_f ? w.forces : nullptr, want_p ? w.pot : nullptr, nullptr, w.upart, w.energy,
                              w.status, st)))
        return rc;
    record(p, st, 7);
    return HSMA_OK;
}

// The stream device work runs on: the plan's stream, or -- for the legacy
// default stream, which cannot be captured -- a private stream ordered after
// the caller's earlier work by an event.
int work_stream(hsma_plan_s *p, cudaStream_t *out)
{
    if (p->stream) {
        *out = p->stream;
        return HSMA_OK;
    }
    if (!p->priv_stream) {
        HSMA_CUDA_TRY(cudaStreamCreateWithFlags(&p->priv_stream, cudaStreamNonBlocking));
        HSMA_CUDA_TRY(cudaEventCreateWithFlags(&p->order_ev, cudaEventDisableTiming));
    }
    HSMA_CUDA_TRY(cudaEventRecord(p->order_ev, (cudaStream_t)0));
    HSMA_CUDA_TRY(cudaStreamWaitEvent(p->priv_stream, p->order_ev, 0));
    *out = p->priv_stream;
    return HSMA_OK;
}

// Device memory of the reusable in-set for systems of n particles.
size_t carve_md(hsma_plan_s *p, long long n, void *base)
{
    const long long nblk = (n + kInsetBlock - 1) / kInsetBlock;
    Carver c(base);
    p->md_cand = c.take<int2>((size_t)n * p->md_nshifts);
    p->md_perm = c.take<int>(n);
    p->md_x0 = c.take<double4_32a>(n);
    p->md_u = c.take<double4_32a>(n);
    p->md_counts = c.take<int>((size_t)p->md_nshifts * nblk);
    p->md_rcounts = c.take<int>((size_t)p->md_nshifts * nblk + 1);  // per block of 256 candidates
    p->md_shifts = c.take<int4>(p->md_nshifts);
    p->md_ns = c.take<long long>(1);
    return align_up(c.off, 256);
}

int ensure_md(hsma_plan_s *p, long long n)
{
    const size_t need = carve_md(p, n, nullptr);
    if (need > p->md_cap) {
        if (p->md_mem) {
            cudaStreamSynchronize(p->stream ? p->stream : p->priv_stream);
            dev_free(p->md_mem);
        }
        p->md_mem = nullptr;
        p->md_cap = 0;
        p->md_valid = false;
        drop_graphs(p);  // the cached graphs hold pointers into the old list
        HSMA_CUDA_TRY(dev_malloc(&p->md_mem, need));
        p->md_cap = need;
        p->md_shifts_dirty = true;
    }
    carve_md(p, n, p->md_mem);
    if (!p->md_ns_host) HSMA_CUDA_TRY(host_malloc(&p->md_ns_host, sizeof(long long)));
    if (p->md_shifts_dirty) {
        HSMA_CUDA_TRY(cudaMemcpy(p->md_shifts, p->md_shift_host.data(), sizeof(int4) * p->md_nshifts,
                                 cudaMemcpyHostToDevice));
        p->md_shifts_dirty = false;
    }
    return HSMA_OK;
}

// Enqueue one update step in the given mode: by replaying a CUDA graph of
// it (captured on first use for this batch shape, mode and buffers) or, with
// graphs off or profiling on, by direct launches.
int launch_step(hsma_plan_s *p, const BatchShape &sh, const Workspace &w, int prec, bool want_f, bool want_p,
                int mode, const std::vector<long long> &n, cudaStream_t st)
{
    if (!(p->use_graphs && !p->profile)) return enqueue_update(p, sh, w, prec, want_f, want_p, mode, st);
    std::vector<long long> key = {prec,
                                  sh.nsys,
                                  want_f,
                                  want_p,
                                  (long long)(uintptr_t)p->ws_mem,
                                  sh.variant,
                                  (long long)sh.items,
                                  mode,
                                  (long long)(uintptr_t)p->md_mem};
    key.insert(key.end(), n.begin(), n.end());
    hsma_plan_s::GraphEntry *g = nullptr;
    for (auto &e : p->graphs)
        if (e.key == key) g = &e;
    if (!g) {
        constexpr size_t kKeep = 3;  // graphs cached per plan
        if (p->graphs.size() >= kKeep) {
            auto old = std::min_element(p->graphs.begin(), p->graphs.end(),
                                        [](const auto &a, const auto &b) { return a.last_use < b.last_use; });
            cudaGraphExecDestroy(old->exec);
            p->graphs.erase(old);
        }
        long long before = g_launches.load();
        HSMA_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_update(p, sh, w, prec, want_f, want_p, mode, st);
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(st, &graph);
        if (rc || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (!rc) set_last_cuda_error(ce, "cudaStreamEndCapture", __FILE__, __LINE__);
            return rc ? rc : HSMA_E_CUDA;
        }
        hsma_plan_s::GraphEntry e;
        ce = cudaGraphInstantiate(&e.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            set_last_cuda_error(ce, "cudaGraphInstantiate", __FILE__, __LINE__);
            return HSMA_E_CUDA;
        }
        e.kernels = g_launches.load() - before;
        g_launches.fetch_sub(e.kernels);  // counted when replayed
        e.key = key;
        p->graphs.push_back(e);
        g = &p->graphs.back();
    }
    g->last_use = ++p->graph_clock;
    HSMA_CUDA_TRY(cudaGraphLaunch(g->exec, st));
    g_launches.fetch_add(g->kernels);
    return HSMA_OK;
}

// The update step for a batch of systems sharing the plan.
int run_update(hsma_plan_s *p, int nsys, const int64_t *offsets, const hsma_particles *all, double *energies,
               double *forces, double *pot, int *status_out, hsma_out *single)
{
    if (!p || nsys < 1 || !offsets || !all || !all->xyz || !all->q) return HSMA_E_ARG;
    if (offsets[0] != 0) return HSMA_E_ARG;
    if (((uintptr_t)all->xyz | (uintptr_t)all->q | (uintptr_t)forces | (uintptr_t)pot) & 7) return HSMA_E_ARG;
    if (nsys > kMaxSystems) return HSMA_E_ARG;
    std::vector<long long> n(nsys);
    for (int s = 0; s < nsys; ++s) {
        n[s] = offsets[s + 1] - offsets[s];
        if (n[s] < 1 || n[s] > kMaxInsetSlots / p->nshifts) return HSMA_E_ARG;
    }
    const int prec = p->precision;
    const bool on_dev = all->on_device != 0;
    BatchShape sh;
    shape_batch(p, nsys, n.data(), prec, choose_tuning(p, nsys, n.data()), &sh);
    if (sh.items < 0 || sh.surf_items < 0 || sh.cap_total > (1LL << 40)) return HSMA_E_ARG;
    Workspace w;
    size_t need = carve_workspace(p, sh, prec, true, true, nullptr, &w);
    int rc = ensure_workspace(p, need);
    if (rc) return rc;
    carve_workspace(p, sh, prec, true, true, p->ws_mem, &w);
    p->ws = w;
    const size_t sys_bytes = align_up(sizeof(SysDesc) * nsys, 64);
    const size_t pin_bytes = sys_bytes + align_up(sizeof(double) * nsys, 64) + align_up(sizeof(long long) * nsys, 64) +
                             align_up(sizeof(int) * nsys, 64);
    rc = ensure_pinned(p, pin_bytes);
    if (rc) return rc;
    SysDesc *hsys = (SysDesc *)p->hpin;
    double *h_energy = (double *)((char *)p->hpin + sys_bytes);
    long long *h_ns = (long long *)((char *)h_energy + align_up(sizeof(double) * nsys, 64));
    int *h_status = (int *)((char *)h_ns + align_up(sizeof(long long) * nsys, 64));
    memcpy(hsys, sh.sys.data(), sizeof(SysDesc) * nsys);
    cudaStream_t st;
    if ((rc = work_stream(p, &st))) return rc;
    const cudaMemcpyKind in_kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind out_kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;

    // inputs into the workspace (outside any graph: the caller's pointers vary)
    HSMA_CUDA_TRY(cudaMemcpyAsync(w.sys, hsys, sizeof(SysDesc) * nsys, cudaMemcpyHostToDevice, st));
    HSMA_CUDA_TRY(cudaMemcpyAsync(w.xyz, all->xyz, sizeof(double) * 3 * sh.n_total, in_kind, st));
    HSMA_CUDA_TRY(cudaMemcpyAsync(w.q, all->q, sizeof(double) * sh.n_total, in_kind, st));

    const bool want_f = forces != nullptr, want_p = pot != nullptr;
    int mode = kFull;
    if (p->md_skin > 0.0 && nsys == 1) {
        if ((rc = ensure_md(p, n[0]))) return rc;
        mode = (p->md_valid && p->md_n == n[0] && p->md_prec == prec) ? kReuse : kBuild;
    }
    auto device_step = [&](int m) -> int {
        int r = launch_step(p, sh, w, prec, want_f, want_p, m, n, st);
        if (r) return r;
        HSMA_CUDA_TRY(cudaMemcpyAsync(h_energy, w.energy, sizeof(double) * nsys, cudaMemcpyDeviceToHost, st));
        HSMA_CUDA_TRY(cudaMemcpyAsync(h_status, w.status, sizeof(int) * nsys, cudaMemcpyDeviceToHost, st));
        HSMA_CUDA_TRY(cudaMemcpyAsync(h_ns, w.ns, sizeof(long long) * nsys, cudaMemcpyDeviceToHost, st));
        if (m == kBuild)
            HSMA_CUDA_TRY(cudaMemcpyAsync(p->md_ns_host, p->md_ns, sizeof(long long), cudaMemcpyDeviceToHost, st));
        if (want_f) HSMA_CUDA_TRY(cudaMemcpyAsync(forces, w.forces, sizeof(double) * 3 * sh.n_total, out_kind, st));
        if (want_p) HSMA_CUDA_TRY(cudaMemcpyAsync(pot, w.pot, sizeof(double) * sh.n_total, out_kind, st));
        HSMA_CUDA_TRY(cudaStreamSynchronize(st));
        HSMA_CUDA_TRY(cudaGetLastError());
        return HSMA_OK;
    };
    if ((rc = device_step(mode))) return rc;
    if (mode == kReuse && (h_status[0] & ST_STALE)) {
        // a particle moved by the skin or more (or the charges changed): the
        // list no longer covers the in-set; redo the step with a new list
        ++p->md_stale;
        p->md_valid = false;
        mode = kBuild;
        if ((rc = device_step(mode))) return rc;
    }
    if (mode == kReuse) ++p->md_reuses;
    if (mode == kBuild) {
        ++p->md_builds;
        p->md_valid = map_status(h_status[0]) == HSMA_OK;
        p->md_n = n[0];
        p->md_ncand = *p->md_ns_host;
        p->md_prec = prec;
    }

    if (p->profile && p->events_ready) {
        const int from[8] = {0, 1, 2, 3, 4, 5, 6, 0};
        const int to[8] = {1, 2, 3, 4, 5, 6, 7, 7};
        for (int i = 0; i < 8; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, p->ev[from[i]], p->ev[to[i]]);
            p->last_ms[i] = ms;
        }
        p->have_timings = true;
    }
    p->last_nsys = nsys;
    p->last_n = sh.n_total;
    p->last_shape = sh;

    int worst = HSMA_OK;
    for (int s = 0; s < nsys; ++s) {
        if (energies) energies[s] = h_energy[s];
        int code = map_status(h_status[s]);
        if (status_out) status_out[s] = code;
        if (code != HSMA_OK && worst == HSMA_OK) worst = code;
    }
    if (single) {
        single->energy = h_energy[0];
        single->n_inset = h_ns[0];
        single->n_images = 6 * (p->F2 + 1);
    }
    return worst;
}

// Morton order of the monitoring targets (a 1024^3 grid over the sphere of
// radius R0 that holds all of them), so that each block of targets the pair
// kernel takes is a compact region and far source tiles skip the low words.
int sort_monitor_targets(hsma_plan_s *p, cudaStream_t st)
{
    const int n = p->nmon;
    std::vector<double4_32a> h(n);
    HSMA_CUDA_TRY(cudaMemcpyAsync(h.data(), p->mon64, sizeof(double4_32a) * n, cudaMemcpyDeviceToHost, st));
    HSMA_CUDA_TRY(cudaStreamSynchronize(st));
    auto spread = [](unsigned v) {
        unsigned long long x = v & 0x3ffu, r = 0;
        for (int b = 0; b < 10; ++b) r |= ((x >> b) & 1ull) << (3 * b);
        return r;
    };
    std::vector<unsigned long long> key(n);
    const double lo = -p->R0 * 1.000001, w = 2.0 * p->R0 * 1.000001;
    for (int i = 0; i < n; ++i) {
        const double c[3] = {h[i].x, h[i].y, h[i].z};
        unsigned cell[3];
        for (int a = 0; a < 3; ++a) {
            double f = (c[a] - lo) / w * 1024.0;
            int k = (int)floor(f);
            cell[a] = (unsigned)std::min(1023, std::max(0, k));
        }
        key[i] = spread(cell[0]) | (spread(cell[1]) << 1) | (spread(cell[2]) << 2);
    }
    p->mon_perm.resize(n);
    for (int i = 0; i < n; ++i) p->mon_perm[i] = i;
    std::stable_sort(p->mon_perm.begin(), p->mon_perm.end(), [&](int a, int b) { return key[a] < key[b]; });
    std::vector<int> inv(n);
    for (int k = 0; k < n; ++k) inv[p->mon_perm[k]] = k;
    HSMA_CUDA_TRY(cudaMemcpyAsync(p->mon_perm_d, p->mon_perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    HSMA_CUDA_TRY(cudaMemcpyAsync(p->mon_inv, inv.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    int rc = launch_gather_targets(n, p->mon_perm_d, p->mon64, p->mon_hi, p->mon_lo, p->mon64_s, p->mon_hi_s,
                                   p->mon_lo_s, st);
    if (rc) return rc;
    rc = launch_array_boxes(n, p->mon_hi_s, pair_targets_per_block(HSMA_FP32_ACC64, 4), p->mon_boxes, st);
    if (rc) return rc;
    rc = launch_array_boxes(n, p->mon_hi_s, pair_targets_per_block(HSMA_FP32_ACC64, 2), p->mon_boxes2, st);
    if (rc) return rc;
    rc = launch_array_boxes(n, p->mon_hi_s, pair_targets_per_block(HSMA_FP32_ACC64, 17), p->mon_boxes3, st);
    if (rc) return rc;
    HSMA_CUDA_TRY(cudaStreamSynchronize(st));  // host vectors above go out of scope
    return HSMA_OK;
}

__global__ void shard_gather_kernel(long long lo, long long cnt, const int *perm, const double *phi_src,
                                    const double *e_src, long long *idx_out, double *phi_out, double *field_out)
{
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cnt) return;
    long long i = lo + j;
    idx_out[j] = perm[i];
    phi_out[j] = phi_src[i];
    field_out[3 * j] = e_src[3 * i];
    field_out[3 * j + 1] = e_src[3 * i + 1];
    field_out[3 * j + 2] = e_src[3 * i + 2];
}

// One stage of the target-sharded update step for part `part` of `nparts`
// (see hsma_shard_near / hsma_shard_far).  Single system; host outputs.
int run_shard(hsma_plan_s *p, const hsma_particles *x, bool far_stage, int part, int nparts,
              const double *phi_mon_in, const double *phi_in, const double *field_in, int64_t count_in,
              double *phi_mon_out, int64_t *index, double *phi, double *field, int64_t *count, double *energy)
{
    if (!p || !x || !x->xyz || !x->q || x->n < 1 || nparts < 1 || part < 0 || part >= nparts || !index || !phi ||
        !field || !count)
        return HSMA_E_ARG;
    if (far_stage ? (!phi_mon_in || !phi_in || !field_in || !energy) : !phi_mon_out) return HSMA_E_ARG;
    const long long n = x->n;
    if (n > kMaxInsetSlots / p->nshifts) return HSMA_E_ARG;
    const int prec = p->precision;
    BatchShape sh;
    shape_batch(p, 1, &n, prec, choose_tuning(p, 1, &n), &sh);
    if (sh.items < 0 || sh.surf_items < 0) return HSMA_E_ARG;
    SysDesc &d = sh.sys[0];
    const int TB = pair_targets_per_block(prec, sh.variant);
    const int STB = surface_targets_per_block();
    const long long nb = (n + TB - 1) / TB, nbm = (p->nmon + TB - 1) / TB;
    const int pb_lo = (int)(part * nb / nparts), pb_hi = (int)((part + 1) * nb / nparts);
    const int mb_lo = (int)(part * nbm / nparts), mb_hi = (int)((part + 1) * nbm / nparts);
    const long long t_lo = std::min<long long>((long long)pb_lo * TB, n);
    const long long t_hi = std::min<long long>((long long)pb_hi * TB, n);
    const long long m_lo = std::min<long long>((long long)mb_lo * TB, p->nmon);
    const long long m_hi = std::min<long long>((long long)mb_hi * TB, p->nmon);
    d.pb_lo = pb_lo;
    d.mb_lo = mb_lo;
    d.ntb_part = pb_hi - pb_lo;
    d.ntb = d.ntb_part + (mb_hi - mb_lo);
    sh.items = d.ntb * d.nchunks;
    d.sp_lo = t_lo;
    d.sp_n = t_hi - t_lo;
    sh.surf_items = (int)((d.sp_n + STB - 1) / STB);

    Workspace w;
    size_t need = carve_workspace(p, sh, prec, true, true, nullptr, &w);
    int rc = ensure_workspace(p, need);
    if (rc) return rc;
    carve_workspace(p, sh, prec, true, true, p->ws_mem, &w);
    p->ws = w;
    if ((rc = ensure_pinned(p, sizeof(SysDesc) + 64))) return rc;
    memcpy(p->hpin, &d, sizeof(SysDesc));
    cudaStream_t st;
    if ((rc = work_stream(p, &st))) return rc;
    const cudaMemcpyKind in_kind = x->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    HSMA_CUDA_TRY(cudaMemcpyAsync(w.sys, p->hpin, sizeof(SysDesc), cudaMemcpyHostToDevice, st));
    HSMA_CUDA_TRY(cudaMemcpyAsync(w.xyz, x->xyz, sizeof(double) * 3 * n, in_kind, st));
    HSMA_CUDA_TRY(cudaMemcpyAsync(w.q, x->q, sizeof(double) * n, in_kind, st));
    HSMA_CUDA_TRY(cudaMemsetAsync(w.status, 0, sizeof(int), st));
    HSMA_CUDA_TRY(cudaMemsetAsync(w.ctrl, 0, sizeof(int) * 8, st));

    // sort and in-set (both stages: the far stage needs the particles in
    // spatial order again)
    SortArgs sa;
    sa.sys = w.sys;
    sa.nsys = 1;
    sa.xyz = w.xyz;
    for (int a = 0; a < 3; ++a) sa.g.L[a] = p->L[a];
    sa.g.Rs = p->Rs;
    sa.g.bc = p->bc;
    sa.keys = w.keys;
    sa.vals = w.perm;
    sa.keys2 = w.keys2;
    sa.vals2 = w.vals2;
    sa.hist = w.hist;
    if ((rc = launch_sort_particles(sa, sh.nblk_max, st))) return rc;
    InsetArgs ia;
    ia.sys = w.sys;
    ia.nsys = 1;
    ia.nblk_max = sh.nblk_max;
    ia.xyz = w.xyz;
    ia.q = w.q;
    ia.perm = w.perm;
    ia.shifts = p->shifts;
    ia.n_shifts = p->nshifts;
    ia.g = sa.g;
    ia.counts = w.counts;
    ia.ns = w.ns;
    ia.src_hi = w.src_hi;
    ia.src_lo = w.src_lo;
    ia.src64 = w.src64;
    ia.status = w.status;
    ia.cen = w.cen;
    ia.cenf = w.cenf;
    ia.qsums = w.qsums;
    if ((rc = launch_inset(ia, st))) return rc;

    const long long cnt = t_hi - t_lo;
    if (far_stage && count_in != cnt) return HSMA_E_ARG;  // not this part's near-stage arrays
    std::vector<double> mon(p->nmon);
    if (!far_stage) {
        if (w.boxes && (rc = launch_tile_boxes(w.sys, 1, sh.max_tiles, w.ns, w.src_hi, TB, w.boxes, st))) return rc;
        PairArgs pa;
        pa.sys = w.sys;
        pa.nsys = 1;
        pa.total_items = sh.items;
        pa.ns = w.ns;
        pa.src_hi = w.src_hi;
        pa.src_lo = w.src_lo;
        pa.src64 = w.src64;
        pa.ext_hi = p->mon_hi_s;
        pa.ext_lo = p->mon_lo_s;
        pa.ext64 = p->mon64_s;
        pa.n_ext = p->nmon;
        pa.ext_field = 0;
        pa.ext_skip_zero = 0;
        pa.boxes = w.boxes;
        pa.ext_boxes = w.boxes ? (TB == 256 ? p->mon_boxes2 : (TB == 384 ? p->mon_boxes3 : p->mon_boxes)) : nullptr;
        pa.far2 = (float)(p->far_rel * p->Rs * p->far_rel * p->Rs);
        pa.partials = w.partials;
        pa.next_item = w.ctrl;
        pa.status = w.status;
        const int grid = std::max(1, std::min(sh.items, p->num_sms * tuned_ctas(p, prec, sh.variant)));
        if ((rc = launch_pair(pa, prec, sh.variant, grid, st))) return rc;
        if ((rc = launch_partial_reduce(w.sys, 1, sh.max_tgt, p->nmon, w.partials, prec, w.phi_tgt, w.e_part, st)))
            return rc;
        if (cnt > 0) {
            shard_gather_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(t_lo, cnt, w.perm, w.phi_tgt,
                                                                                w.e_part, w.idx64, w.pot, w.forces);
            HSMA_LAUNCHED();
        }
        HSMA_CUDA_TRY(cudaMemcpyAsync(mon.data(), w.phi_tgt + n, sizeof(double) * p->nmon, cudaMemcpyDeviceToHost,
                                      st));
    } else {
        // the full monitoring potentials, into the spatially ordered slots
        for (int k = 0; k < p->nmon; ++k) mon[k] = phi_mon_in[p->mon_perm[k]];
        HSMA_CUDA_TRY(cudaMemcpyAsync(w.phi_tgt + n, mon.data(), sizeof(double) * p->nmon, cudaMemcpyHostToDevice,
                                      st));
        if (prec == HSMA_FP32_TC_FIT)
            rc = launch_fit_tc(w.sys, 1, p->bc, p->K, p->ncols, p->Nb, p->tc_hi, p->tc_lo, p->tc_mdf, w.phi_tgt,
                               p->mon_inv, w.b, w.A, w.tc_work, w.status, fit_ctas(p), st);
        else
            rc = launch_fit_fp64(w.sys, 1, p->bc, p->K, p->ncols, p->Nb, p->Mp, w.phi_tgt, p->mon_inv, w.b, w.A, st);
        if (rc) return rc;
        if (p->far_field == 1) {
            rc = launch_series_field(w.sys, 1, std::max<long long>(cnt, 1), p->P, p->Rs, p->norm, w.A, w.src_hi,
                                     w.src_lo, w.src64, w.phi_out, w.e_out, st);
        } else {
            rc = launch_surface_charges(1, p->ndir, p->Nb, p->Bq, p->dirs, w.A, p->Rs, w.img, st);
            if (!rc && sh.surf_items > 0)
                rc = launch_surface_pairs(w.sys, 1, sh.surf_items, w.ns, w.src_hi, w.src_lo, w.src64, p->ndir,
                                          p->dirs, w.img, p->Rs, p->dr, prec, w.phi_out, w.e_out, st);
        }
        if (rc) return rc;
        // the near stage's Phi_in, E_in of the owned particles into their
        // target slots, then potentials, forces and the part's energy
        // 1/2 sum q_i (Phi_in + Phi_out) on the device (owned order)
        if (cnt > 0) {
            HSMA_CUDA_TRY(cudaMemcpyAsync(w.phi_tgt + t_lo, phi_in, sizeof(double) * cnt, cudaMemcpyHostToDevice,
                                          st));
            HSMA_CUDA_TRY(cudaMemcpyAsync(w.e_part + 3 * t_lo, field_in, sizeof(double) * 3 * cnt,
                                          cudaMemcpyHostToDevice, st));
        }
        if ((rc = launch_finalize(w.sys, 1, std::max<long long>(cnt, 1), w.perm, w.q, w.phi_tgt, w.e_part,
                                  w.phi_out, w.e_out, w.forces, w.pot, w.idx64, w.upart, w.energy, w.status, st)))
            return rc;
    }
    std::vector<long long> idx(std::max<long long>(cnt, 1));
    int hst = 0;
    double u_part = 0.0;
    if (cnt > 0) {
        HSMA_CUDA_TRY(cudaMemcpyAsync(idx.data(), w.idx64, sizeof(long long) * cnt, cudaMemcpyDeviceToHost, st));
        HSMA_CUDA_TRY(cudaMemcpyAsync(phi, w.pot, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
        HSMA_CUDA_TRY(cudaMemcpyAsync(field, w.forces, sizeof(double) * 3 * cnt, cudaMemcpyDeviceToHost, st));
    }
    if (far_stage) HSMA_CUDA_TRY(cudaMemcpyAsync(&u_part, w.energy, sizeof(double), cudaMemcpyDeviceToHost, st));
    HSMA_CUDA_TRY(cudaMemcpyAsync(&hst, w.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    HSMA_CUDA_TRY(cudaStreamSynchronize(st));
    HSMA_CUDA_TRY(cudaGetLastError());
    for (long long j = 0; j < cnt; ++j) index[j] = idx[j];
    *count = cnt;
    if (far_stage) *energy = u_part;
    if (!far_stage) {
        for (int k = 0; k < p->nmon; ++k) phi_mon_out[k] = 0.0;
        for (long long k = m_lo; k < m_hi; ++k) phi_mon_out[p->mon_perm[k]] = mon[k];
    }
    p->last_nsys = 0;  // the workspace no longer holds a whole-system result
    return map_status(hst);
}

std::mutex g_scratch_mu;

// Everything a plan's parameters fix before any device work: the checked
// options and the derived sizes (basis, fitted columns, monitoring targets,
// Fibonacci rule, image shells, Delta r).  Pure host arithmetic; shared by
// hsma_plan and hsma_plan_dims.
struct PlanParams {
    hsma_opts o;
    double R0, dr;
    int Nb, ncols, nmon, F2, F1, Ks[3], nshifts;
};

int plan_params(const double box[3], int bc, int p, double R, int Q, int Kmon, const hsma_opts *opts,
                PlanParams *pp)
{
    hsma_opts o;
    hsma_opts_default(&o);
    if (opts) o = *opts;
    if (!(box[0] > 0 && box[1] > 0 && box[2] > 0)) return HSMA_E_ARG;
    if (bc != HSMA_BC_PERIODIC && bc != HSMA_BC_GROUNDED) return HSMA_E_ARG;
    if (p < 1 || p > 40) return HSMA_E_ARG;
    if (o.precision < 0 || o.precision > 2) return HSMA_E_ARG;
    if (o.far_field != 0 && o.far_field != 1) return HSMA_E_ARG;
    const double R0 = 0.5 * sqrt(box[0] * box[0] + box[1] * box[1] + box[2] * box[2]);
    if (!(R > R0) || !isfinite(R)) return HSMA_E_ARG;
    const int Nb = (p + 1) * (p + 1);
    const int ncols = (bc == HSMA_BC_PERIODIC) ? Nb - 1 : Nb;
    if (Kmon < ncols || Kmon > 16384) return HSMA_E_ARG;
    int F2 = 0, F1 = 0;
    if (o.fib_F2 > 0) {
        F2 = o.fib_F2;
        if (!fib_pred(F2, &F1) || F2 < 2) return HSMA_E_ARG;
    } else {
        if (Q < 12) return HSMA_E_ARG;
        fib_from_q(Q, &F2, &F1);
    }
    long long nsh = 1;
    for (int a = 0; a < 3; ++a) {
        pp->Ks[a] = shells(R, box[a]);
        nsh *= 2LL * pp->Ks[a] + 1;
    }
    if (nsh > kMaxShifts) return HSMA_E_ARG;  // sphere too large for the box
    pp->o = o;
    pp->R0 = R0;
    pp->dr = (o.dr_rel > 0 ? o.dr_rel : (bc == HSMA_BC_PERIODIC ? 1e-5 : 1e-4)) * R;
    pp->Nb = Nb;
    pp->ncols = ncols;
    pp->nmon = (bc == HSMA_BC_PERIODIC) ? 2 * Kmon : Kmon;
    pp->F2 = F2;
    pp->F1 = F1;
    pp->nshifts = (int)nsh;
    return HSMA_OK;
}

}  // namespace

int hsma::plan_reserve(hsma_plan_t p, int nsys, long long n_each)
{
    if (!p || nsys < 1 || nsys > kMaxSystems || n_each < 1 || n_each > kMaxInsetSlots / p->nshifts)
        return HSMA_E_ARG;
    // the largest workspace over the batch and the single request of that
    // size: they take different tunings (and so tiles and work items)
    size_t need = 0;
    for (int k : {1, nsys}) {
        std::vector<long long> n(k, n_each);
        BatchShape sh;
        shape_batch(p, k, n.data(), p->precision, choose_tuning(p, k, n.data()), &sh);
        if (sh.items < 0 || sh.surf_items < 0) return HSMA_E_ARG;
        Workspace w;
        need = std::max(need, carve_workspace(p, sh, p->precision, true, true, nullptr, &w));
    }
    int rc = ensure_workspace(p, need);
    if (rc) return rc;
    const size_t pin_bytes = align_up(sizeof(SysDesc) * nsys, 64) + align_up(sizeof(double) * nsys, 64) +
                             align_up(sizeof(long long) * nsys, 64) + align_up(sizeof(int) * nsys, 64);
    return ensure_pinned(p, pin_bytes);
}

void hsma::plan_trim_workspace(hsma_plan_t p, size_t max_keep)
{
    if (!p || p->ws_cap <= max_keep || !p->ws_mem) return;
    cudaStream_t st = p->stream ? p->stream : p->priv_stream;
    if (st) cudaStreamSynchronize(st);
    drop_graphs(p);
    dev_free(p->ws_mem);
    p->ws_mem = nullptr;
    p->ws_cap = 0;
    p->ws = Workspace();
    p->last_nsys = 0;
}

extern "C" {

int hsma_opts_default(hsma_opts *o)
{
    if (!o) return HSMA_E_ARG;
    memset(o, 0, sizeof(*o));
    o->precision = HSMA_FP32_ACC64;
    o->dr_rel = 0.0;
    o->fib_F2 = 0;
    o->far_field = 0;
    o->stream = nullptr;
    o->use_graphs = 1;
    o->profile = 0;
    return HSMA_OK;
}

const char *hsma_version(void) { return "hsma-gb300 0.1 (sm_103a)"; }

const char *hsma_strerror(int code)
{
    switch (code) {
        case HSMA_OK: return "ok";
        case HSMA_E_ARG: return "invalid argument";
        case HSMA_E_NONNEUTRAL: return "periodic system is not charge neutral";
        case HSMA_E_OUT_OF_BOX: return "particle outside the grounded box, on a wall, or not finite";
        case HSMA_E_COINCIDENT: return "coincident charges (non-finite result)";
        case HSMA_E_OOM: return "out of memory";
        case HSMA_E_TIMEOUT: return "bounded device wait timed out";
        case HSMA_E_CUDA: return g_cuda_err[0] ? g_cuda_err : "CUDA error";
        case HSMA_E_ILLCOND: return "fitting matrix is numerically rank deficient";
        case HSMA_E_NOT_FOUND: return "not found";
        case HSMA_E_AGAIN: return "not ready";
        case HSMA_E_CAPACITY: return "request exceeds the memory budget (serving) or the static scratch array";
        case HSMA_E_CANCELLED: return "request cancelled";
        default: return "unknown error";
    }
}

int64_t hsma_kernel_launches(void) { return g_launches.load(); }

int64_t hsma_allocation_calls(void) { return g_alloc_calls.load(); }

int hsma_plan(hsma_plan_t *out, const double box[3], int bc, int p, double R, int Q, int Kmon, const hsma_opts *opts)
{
    if (!out || !box) return HSMA_E_ARG;
    *out = nullptr;
    PlanParams pp;
    if (int e = plan_params(box, bc, p, R, Q, Kmon, opts, &pp)) return e;
    const hsma_opts &o = pp.o;
    const double R0 = pp.R0;
    const int Nb = pp.Nb, ncols = pp.ncols, F2 = pp.F2, F1 = pp.F1;

    hsma_plan_s *pl = new hsma_plan_s();
    for (int a = 0; a < 3; ++a) pl->L[a] = box[a];
    pl->bc = bc;
    pl->P = p;
    pl->Nb = Nb;
    pl->ncols = ncols;
    pl->K = Kmon;
    pl->mon_faces = (bc == HSMA_BC_GROUNDED) ? 1 : 0;
    pl->nmon = pp.nmon;
    pl->F2 = F2;
    pl->F1 = F1;
    pl->ndir = 2 * (F2 + 1);
    pl->Rs = R;
    pl->R0 = R0;
    pl->alpha = R / R0;
    pl->dr = pp.dr;
    pl->precision = o.precision;
    pl->use_graphs = o.use_graphs;
    pl->profile = o.profile;
    pl->stream = (cudaStream_t)o.stream;
    pl->far_field = o.far_field;
    {
        const char *e = getenv("HSMA_TEST_STALL_WAIT");
        pl->stall_test = (e && e[0] == '1') ? 1 : 0;
    }

    int rc = HSMA_OK;
    auto fail = [&](int code) {
        hsma_plan_destroy(pl);
        return code;
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(HSMA_E_CUDA);
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return fail(HSMA_E_CUDA);
    pl->num_sms = prop.multiProcessorCount;
    pl->ctas[0] = pair_max_ctas_per_sm(HSMA_FP64);
    pl->ctas[1] = pl->ctas[2] = pair_max_ctas_per_sm(HSMA_FP32_ACC64, 4);
    for (int v = 1; v < hsma_plan_s::kVariantCodes; ++v)
        if (pair_variant_valid(v)) pl->ctas_var[v] = pair_max_ctas_per_sm(HSMA_FP32_ACC64, v);
    snprintf(pl->device_name, sizeof(pl->device_name), "%s", prop.name);

    // image shift table: k = 0 first, then lexicographic (kx, ky, kz)
    const int *Ks = pp.Ks;
    std::vector<int4> sh;
    sh.push_back(make_int4(0, 0, 0, 0));
    for (int kx = -Ks[0]; kx <= Ks[0]; ++kx)
        for (int ky = -Ks[1]; ky <= Ks[1]; ++ky)
            for (int kz = -Ks[2]; kz <= Ks[2]; ++kz) {
                if (!kx && !ky && !kz) continue;
                sh.push_back(make_int4(kx, ky, kz, (abs(kx) + abs(ky) + abs(kz)) & 1));
            }
    pl->nshifts = (int)sh.size();

    // plan memory
    const int K = Kmon, nmon = pl->nmon, ndir = pl->ndir;
    Carver c(nullptr);
    for (int pass = 0; pass < 2; ++pass) {
        c = Carver(pl->plan_mem);
        pl->mon64 = c.take<double4_32a>(nmon);
        pl->mon_hi = c.take<float4>(nmon);
        pl->mon_lo = c.take<float4>(nmon);
        pl->mon64_s = c.take<double4_32a>(nmon);
        pl->mon_hi_s = c.take<float4>(nmon);
        pl->mon_lo_s = c.take<float4>(nmon);
        pl->mon_boxes = c.take<float4>(2 * ((nmon + 255) / 256 + 1));
        pl->mon_boxes2 = c.take<float4>(2 * ((nmon + 255) / 256 + 1));
        pl->mon_boxes3 = c.take<float4>(2 * ((nmon + 255) / 256 + 1));
        pl->mon_perm_d = c.take<int>(nmon);
        pl->mon_inv = c.take<int>(nmon);
        pl->Mrow = c.take<double>((size_t)K * ncols);
        pl->Mp = c.take<double>((size_t)ncols * K);
        pl->dirs = c.take<double4_32a>(ndir);
        pl->Bq = c.take<double>((size_t)ndir * Nb);
        pl->norm = c.take<double>(Nb);
        pl->shifts = c.take<int4>(sh.size());
        pl->tc_hi = c.take<char>(tc_operand_bytes(K, ncols));
        pl->tc_lo = c.take<char>(tc_operand_bytes(K, ncols));
        pl->tc_mdf = c.take<char>(tc_residual_matrix_bytes(K, ncols));
        if (pass == 0) {
            if (dev_malloc(&pl->plan_mem, align_up(c.off, 256)) != cudaSuccess) {
                cudaGetLastError();
                return fail(HSMA_E_OOM);
            }
        }
    }
    // temporaries for the basis at monitoring points and the column-major M
    double *Bx = nullptr, *Mcol = nullptr;
    size_t tmp_bytes = sizeof(double) * ((size_t)nmon * Nb + (size_t)K * ncols);
    if (dev_malloc(&Bx, tmp_bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(HSMA_E_OOM);
    }
    Mcol = Bx + (size_t)nmon * Nb;
    cudaStream_t st = pl->stream;
    auto nt = norm_table(p);
    int rank_ok = 1;
    double cond = 0.0;
    do {
        if (cudaMemcpyAsync(pl->norm, nt.data(), sizeof(double) * Nb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(pl->shifts, sh.data(), sizeof(int4) * sh.size(), cudaMemcpyHostToDevice, st) !=
                cudaSuccess) {
            rc = HSMA_E_CUDA;
            break;
        }
        if (!pl->mon_faces) {
            rc = launch_monitor_sphere(K, R0, box, pl->mon64, pl->mon_hi, pl->mon_lo, st);
        } else {
            // K points over the six faces in proportion to area (largest remainder)
            double area[6], tot = 0;
            for (int f = 0; f < 6; ++f) {
                int a = f / 2;
                area[f] = box[(a + 1) % 3] * box[(a + 2) % 3];
                tot += area[f];
            }
            int cnt[6], used = 0;
            double frac[6];
            for (int f = 0; f < 6; ++f) {
                double quota = K * area[f] / tot;
                cnt[f] = (int)floor(quota);
                frac[f] = quota - cnt[f];
                used += cnt[f];
            }
            while (used < K) {
                int best = 0;
                for (int f = 1; f < 6; ++f)
                    if (frac[f] > frac[best]) best = f;
                cnt[best]++;
                frac[best] = -1.0;
                used++;
            }
            rc = launch_monitor_faces(cnt, box, pl->mon64, pl->mon_hi, pl->mon_lo, st);
        }
        if (rc) break;
        // basis at the monitoring targets (stride 4 doubles per point)
        if ((rc = launch_basis(p, R, nmon, (const double *)pl->mon64, 4, Bx, Nb, st))) break;
        const double *Bxt = (bc == HSMA_BC_PERIODIC) ? Bx + (size_t)K * Nb : nullptr;
        if ((rc = launch_fitting_matrix(K, Nb, ncols, bc == HSMA_BC_PERIODIC ? 1 : 0, Bx, Bxt, Mcol, pl->Mrow, st)))
            break;
        if ((rc = build_pseudo_inverse(K, ncols, Mcol, pl->Mp, &cond, &rank_ok, st))) break;
        if ((rc = launch_quadrature(F2, F1, R, pl->dirs, st))) break;
        // basis at Rs u_j == basis of the unit vector u_j with unit radius
        if ((rc = launch_basis(p, 1.0, ndir, (const double *)pl->dirs, 4, pl->Bq, Nb, st))) break;
        if ((rc = prepare_tc_operands(K, ncols, pl->Mp, pl->Mrow, pl->tc_hi, pl->tc_lo, pl->tc_mdf, st))) break;
        if ((rc = sort_monitor_targets(pl, st))) break;
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            rc = HSMA_E_CUDA;
            break;
        }
    } while (0);
    dev_free(Bx);
    if (rc) return fail(rc);
    pl->cond = cond;
    if (!rank_ok || !(cond < 1e15)) return fail(HSMA_E_ILLCOND);
    if (pl->profile) {
        for (int i = 0; i < 8; ++i)
            if (cudaEventCreate(&pl->ev[i]) != cudaSuccess) return fail(HSMA_E_CUDA);
        pl->events_ready = true;
    }
    *out = pl;
    return HSMA_OK;
}

void hsma_plan_destroy(hsma_plan_t pl)
{
    if (!pl) return;
    if (pl->stream || pl->ws_mem || pl->plan_mem) cudaStreamSynchronize(pl->stream);
    if (pl->priv_stream) cudaStreamSynchronize(pl->priv_stream);
    drop_graphs(pl);
    if (pl->md_mem) dev_free(pl->md_mem);
    if (pl->md_ns_host) host_free(pl->md_ns_host);
    if (pl->priv_stream) cudaStreamDestroy(pl->priv_stream);
    if (pl->order_ev) cudaEventDestroy(pl->order_ev);
    if (pl->events_ready)
        for (int i = 0; i < 8; ++i) cudaEventDestroy(pl->ev[i]);
    if (pl->ws_mem) dev_free(pl->ws_mem);
    if (pl->plan_mem) dev_free(pl->plan_mem);
    if (pl->hpin) host_free(pl->hpin);
    cudaGetLastError();
    delete pl;
}

int hsma_plan_get_info(hsma_plan_t pl, hsma_plan_info_t *info)
{
    if (!pl || !info) return HSMA_E_ARG;
    info->bc = pl->bc;
    info->p = pl->P;
    info->n_basis = pl->Nb;
    info->n_cols = pl->ncols;
    info->Kmon = pl->K;
    info->n_mon_targets = pl->nmon;
    info->F2 = pl->F2;
    info->F1 = pl->F1;
    info->n_images = 6 * (pl->F2 + 1);
    info->n_shifts = pl->nshifts;
    info->Rs = pl->Rs;
    info->R0 = pl->R0;
    info->alpha = pl->alpha;
    info->dr = pl->dr;
    info->cond_estimate = pl->cond;
    info->precision = pl->precision;
    return HSMA_OK;
}

int hsma_plan_dims(const double box[3], int bc, int p, double R, int Q, int Kmon, const hsma_opts *opts,
                   hsma_plan_info_t *info)
{
    if (!box || !info) return HSMA_E_ARG;
    PlanParams pp;
    if (int e = plan_params(box, bc, p, R, Q, Kmon, opts, &pp)) return e;
    info->bc = bc;
    info->p = p;
    info->n_basis = pp.Nb;
    info->n_cols = pp.ncols;
    info->Kmon = Kmon;
    info->n_mon_targets = pp.nmon;
    info->F2 = pp.F2;
    info->F1 = pp.F1;
    info->n_images = 6 * (pp.F2 + 1);
    info->n_shifts = pp.nshifts;
    info->Rs = R;
    info->R0 = pp.R0;
    info->alpha = R / pp.R0;
    info->dr = pp.dr;
    info->cond_estimate = 0.0;
    info->precision = pp.o.precision;
    return HSMA_OK;
}

int hsma_plan_set_stream(hsma_plan_t pl, void *stream)
{
    if (!pl) return HSMA_E_ARG;
    cudaStreamSynchronize(pl->stream);
    pl->stream = (cudaStream_t)stream;
    return HSMA_OK;
}

int hsma_plan_set_precision(hsma_plan_t pl, int precision)
{
    if (!pl || precision < 0 || precision > 2) return HSMA_E_ARG;
    pl->precision = precision;
    return HSMA_OK;
}

int hsma_plan_set_inset_skin(hsma_plan_t pl, double skin)
{
    if (!pl || !(skin >= 0.0)) return HSMA_E_ARG;
    const double lmin = std::min(pl->L[0], std::min(pl->L[1], pl->L[2]));
    // a particle displaced by less than the skin must stay inside the sphere
    // (Rs - R0 is the margin of the box's corners) and within half a box of
    // its build position (the minimum image of the displacement)
    if (skin > 0.0 && !(skin < pl->Rs - pl->R0 && 2.0 * skin < lmin)) return HSMA_E_ARG;
    if (skin > 0.0) {
        // shells of the candidates' sphere Rs + skin
        int K[3];
        long long nsh = 1;
        for (int a = 0; a < 3; ++a) {
            K[a] = shells(pl->Rs + skin, pl->L[a]);
            nsh *= 2LL * K[a] + 1;
        }
        if (nsh > kMaxShifts) return HSMA_E_ARG;
        // the plan's own shifts first, in their order (the in-set of a reused
        // step then has the order, and the tiles, of a fresh one), then the
        // shifts only the larger sphere needs
        std::vector<int4> sh;
        int Kp[3];
        for (int a = 0; a < 3; ++a) Kp[a] = shells(pl->Rs, pl->L[a]);
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 0) sh.push_back(make_int4(0, 0, 0, 0));
            for (int kx = -K[0]; kx <= K[0]; ++kx)
                for (int ky = -K[1]; ky <= K[1]; ++ky)
                    for (int kz = -K[2]; kz <= K[2]; ++kz) {
                        if (!kx && !ky && !kz) continue;
                        const bool own = abs(kx) <= Kp[0] && abs(ky) <= Kp[1] && abs(kz) <= Kp[2];
                        if (own == (pass == 0))
                            sh.push_back(make_int4(kx, ky, kz, (abs(kx) + abs(ky) + abs(kz)) & 1));
                    }
        }
        pl->md_shift_host = sh;
        pl->md_nshifts = (int)sh.size();
        pl->md_shifts_dirty = true;
    }
    pl->md_skin = skin;
    pl->md_valid = false;
    return HSMA_OK;
}

int hsma_plan_set_preemptible(hsma_plan_t pl, int on)
{
    if (!pl || (on != 0 && on != 1)) return HSMA_E_ARG;
    if (pl->preemptible != on) {
        cudaStreamSynchronize(pl->stream ? pl->stream : pl->priv_stream);
        drop_graphs(pl);  // the captured launches change shape
        pl->preemptible = on;
    }
    return HSMA_OK;
}

int hsma_plan_inset_stats(hsma_plan_t pl, int64_t *builds, int64_t *reuses, int64_t *stale)
{
    if (!pl) return HSMA_E_ARG;
    if (builds) *builds = pl->md_builds;
    if (reuses) *reuses = pl->md_reuses;
    if (stale) *stale = pl->md_stale;
    return HSMA_OK;
}

int hsma_plan_footprint(hsma_plan_t pl, int64_t n, size_t *bytes)
{
    if (!pl || !bytes || n < 1) return HSMA_E_ARG;
    BatchShape sh;
    long long nn = n;
    shape_batch(pl, 1, &nn, pl->precision, choose_tuning(pl, 1, &nn), &sh);
    Workspace w;
    *bytes = carve_workspace(pl, sh, pl->precision, true, true, nullptr, &w);
    return HSMA_OK;
}

int hsma_plan_get_matrix(hsma_plan_t pl, int which, double *host_out, int64_t count)
{
    if (!pl || !host_out) return HSMA_E_ARG;
    std::vector<double> tmp;
    const void *src = nullptr;
    size_t nd = 0;
    switch (which) {
        case 0: nd = (size_t)pl->nmon * 4; src = pl->mon64; break;
        case 1: nd = (size_t)pl->K * pl->ncols; src = pl->Mrow; break;
        case 2: nd = (size_t)pl->ncols * pl->K; src = pl->Mp; break;
        case 3:
        case 4: nd = (size_t)pl->ndir * 4; src = pl->dirs; break;
        case 5: nd = (size_t)pl->ndir * pl->Nb; src = pl->Bq; break;
        default: return HSMA_E_ARG;
    }
    tmp.resize(nd);
    HSMA_CUDA_TRY(cudaStreamSynchronize(pl->stream));
    HSMA_CUDA_TRY(cudaMemcpy(tmp.data(), src, nd * sizeof(double), cudaMemcpyDeviceToHost));
    if (which == 0 || which == 3) {
        size_t np = nd / 4;
        if ((int64_t)(np * 3) > count) return HSMA_E_ARG;
        for (size_t i = 0; i < np; ++i)
            for (int a = 0; a < 3; ++a) host_out[3 * i + a] = tmp[4 * i + a];
    } else if (which == 4) {
        size_t np = nd / 4;
        if ((int64_t)np > count) return HSMA_E_ARG;
        for (size_t i = 0; i < np; ++i) host_out[i] = tmp[4 * i + 3];
    } else {
        if ((int64_t)nd > count) return HSMA_E_ARG;
        memcpy(host_out, tmp.data(), nd * sizeof(double));
    }
    return HSMA_OK;
}

int hsma_energy_forces(hsma_plan_t pl, const hsma_particles *x, hsma_out *out)
{
    if (!pl || !x || !out || x->n < 1) return HSMA_E_ARG;
    int64_t off[2] = {0, x->n};
    double e = 0.0;
    int rc = run_update(pl, 1, off, x, &e, out->forces, out->potentials, nullptr, out);
    return rc;
}

int hsma_energy_forces_batched(hsma_plan_t pl, int nsys, const int64_t *offsets, const hsma_particles *all,
                               double *energies, double *forces, double *potentials, int *status)
{
    if (!pl || !all || nsys < 1 || !offsets || !energies) return HSMA_E_ARG;
    for (int s = 0; s < nsys; ++s)
        if (offsets[s + 1] <= offsets[s]) return HSMA_E_ARG;
    if (all->n != 0 && all->n != offsets[nsys]) return HSMA_E_ARG;
    return run_update(pl, nsys, offsets, all, energies, forces, potentials, status, nullptr);
}

int hsma_last_timings(hsma_plan_t pl, double *ms, int n)
{
    if (!pl || !ms || n < 0) return HSMA_E_ARG;
    if (!pl->have_timings) return 0;
    int k = std::min(n, 8);
    for (int i = 0; i < k; ++i) ms[i] = pl->last_ms[i];
    return k;
}

int64_t hsma_last_get(hsma_plan_t pl, int which, double *host_out, int64_t count)
{
    if (!pl || !host_out || pl->last_nsys < 1) return HSMA_E_ARG;
    const SysDesc &sd = pl->last_shape.sys[0];
    const double *src = nullptr;
    int64_t nd = 0;
    switch (which) {
        case 0: src = pl->ws.A; nd = pl->Nb; break;
        case 1: src = pl->ws.b; nd = pl->K; break;
        case 2: src = pl->ws.phi_tgt + sd.tgt_off + sd.n; nd = pl->nmon; break;
        case 3: src = pl->ws.phi_tgt + sd.tgt_off; nd = sd.n; break;
        case 4: src = pl->ws.phi_out + sd.part_off; nd = sd.n; break;
        default: return HSMA_E_ARG;
    }
    if (nd > count) return HSMA_E_ARG;
    HSMA_CUDA_TRY(cudaStreamSynchronize(pl->stream));
    if (which == 2) {
        std::vector<double> v(nd);
        HSMA_CUDA_TRY(cudaMemcpy(v.data(), src, nd * sizeof(double), cudaMemcpyDeviceToHost));
        for (int64_t k = 0; k < nd; ++k) host_out[pl->mon_perm[k]] = v[k];
        return nd;
    }
    if (which == 3 || which == 4) {
        // particle values are held in spatial order; return them in caller order
        std::vector<double> v(nd);
        std::vector<int> perm(nd);
        HSMA_CUDA_TRY(cudaMemcpy(v.data(), src, nd * sizeof(double), cudaMemcpyDeviceToHost));
        HSMA_CUDA_TRY(cudaMemcpy(perm.data(), pl->ws.perm + sd.part_off, nd * sizeof(int), cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < nd; ++i) host_out[perm[i]] = v[i];
        return nd;
    }
    HSMA_CUDA_TRY(cudaMemcpy(host_out, src, nd * sizeof(double), cudaMemcpyDeviceToHost));
    return nd;
}

// --------------------------------------------------------- target sharding
int hsma_shard_near(hsma_plan_t pl, const hsma_particles *x, int part, int nparts, int64_t *index, double *phi,
                    double *field, int64_t *count, double *phi_mon)
{
    return run_shard(pl, x, false, part, nparts, nullptr, nullptr, nullptr, 0, phi_mon, index, phi, field, count,
                     nullptr);
}

int hsma_shard_far(hsma_plan_t pl, const hsma_particles *x, const double *phi_mon, const double *phi_in,
                   const double *field_in, int64_t count_in, int part, int nparts, int64_t *index, double *pot,
                   double *forces, int64_t *count, double *energy)
{
    return run_shard(pl, x, true, part, nparts, phi_mon, phi_in, field_in, count_in, nullptr, index, pot, forces,
                     count, energy);
}

// ------------------------------------------------------------------ tuning
int hsma_plan_set_tuning(hsma_plan_t pl, const hsma_tuning *t)
{
    if (!pl) return HSMA_E_ARG;
    if (!t) {
        pl->tune_fixed = false;
        return HSMA_OK;
    }
    if (!pair_variant_valid(t->pair_variant) || t->items_per_slot < 1 ||
        t->items_per_slot > 4096)
        return HSMA_E_ARG;
    pl->tune_fixed = true;
    pl->tune_value = *t;
    return HSMA_OK;
}

int hsma_plan_get_tuning(hsma_plan_t pl, int nsys, const int64_t *offsets, hsma_tuning *out)
{
    if (!pl || !out || nsys < 1 || !offsets) return HSMA_E_ARG;
    std::vector<long long> n(nsys);
    for (int s = 0; s < nsys; ++s) n[s] = offsets[s + 1] - offsets[s];
    *out = choose_tuning(pl, nsys, n.data());
    return HSMA_OK;
}

int hsma_autotune(hsma_plan_t pl, int nsys, const int64_t *offsets, const hsma_particles *all,
                  const char *cache_path, hsma_tuning *best)
{
    if (!pl || nsys < 1 || !offsets || !all) return HSMA_E_ARG;
    std::vector<long long> n(nsys);
    for (int s = 0; s < nsys; ++s) n[s] = offsets[s + 1] - offsets[s];
    const bool fixed0 = pl->tune_fixed;
    const hsma_tuning value0 = pl->tune_value;
    std::vector<double> energies(nsys);
    std::vector<hsma_tuning> cands;
    // candidates: the packed variants and the two-target scalar loop for
    // reference (4, 5, 15, 16 never won on this part; they stay selectable)
    const int variants[5] = {14, 17, 12, 13, 2};
    const int items[4] = {8, 16, 24, 48};
    for (int v = 0; v < (pl->precision == HSMA_FP64 ? 1 : 5); ++v)
        for (int i : items) cands.push_back(hsma_tuning{variants[v], i, 0.0});
    hsma_tuning win{14, 48, 1e300};
    int rc = HSMA_OK;
    for (auto &c : cands) {
        pl->tune_fixed = true;
        pl->tune_value = c;
        double t_best = 1e300;
        for (int rep = 0; rep < 3 && !rc; ++rep) {
            auto t0 = std::chrono::steady_clock::now();
            rc = run_update(pl, nsys, offsets, all, energies.data(), nullptr, nullptr, nullptr, nullptr);
            double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (rep > 0) t_best = std::min(t_best, ms);  // rep 0 warms the workspace and graph
        }
        if (rc) break;
        c.ms = t_best;
        if (t_best < win.ms) win = c;
    }
    pl->tune_fixed = fixed0;
    pl->tune_value = value0;
    if (rc) return rc;
    const int bucket = work_bucket(batch_work(pl, nsys, n.data()));
    bool replaced = false;
    for (auto &e : pl->tune_entries)
        if (e.first == bucket) {
            e.second = win;
            replaced = true;
        }
    if (!replaced) pl->tune_entries.push_back({bucket, win});
    if (best) *best = win;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (!f) return HSMA_E_ARG;
        fprintf(f,
                "{\"device\":\"%s\",\"bc\":%d,\"p\":%d,\"Kmon\":%d,\"F2\":%d,\"precision\":%d,"
                "\"bucket\":%d,\"pair_variant\":%d,\"items_per_slot\":%d,\"ms\":%.4f}\n",
                pl->device_name, pl->bc, pl->P, pl->K, pl->F2, pl->precision, bucket, win.pair_variant,
                win.items_per_slot, win.ms);
        fclose(f);
    }
    return HSMA_OK;
}

int hsma_plan_load_tuning(hsma_plan_t pl, const char *cache_path)
{
    if (!pl || !cache_path) return HSMA_E_ARG;
    FILE *f = fopen(cache_path, "r");
    if (!f) return 0;
    char line[1024], dev[256];
    int loaded = 0;
    while (fgets(line, sizeof(line), f)) {
        int bc, P, K, F2, prec, bucket, var, ips;
        double ms;
        int got = sscanf(line,
                         "{\"device\":\"%255[^\"]\",\"bc\":%d,\"p\":%d,\"Kmon\":%d,\"F2\":%d,\"precision\":%d,"
                         "\"bucket\":%d,\"pair_variant\":%d,\"items_per_slot\":%d,\"ms\":%lf}",
                         dev, &bc, &P, &K, &F2, &prec, &bucket, &var, &ips, &ms);
        if (got != 10) continue;
        if (strcmp(dev, pl->device_name) || bc != pl->bc || P != pl->P || K != pl->K || F2 != pl->F2 ||
            prec != pl->precision || !pair_variant_valid(var) || ips < 1)
            continue;
        bool replaced = false;
        for (auto &e : pl->tune_entries)
            if (e.first == bucket) {
                e.second = hsma_tuning{var, ips, ms};
                replaced = true;
            }
        if (!replaced) pl->tune_entries.push_back({bucket, hsma_tuning{var, ips, ms}});
        ++loaded;
    }
    fclose(f);
    return loaded;
}

// -------------------------------------------------------------- direct sums
namespace {
__global__ void split_sources_kernel(long long n, const double *src, float4 *hi, float4 *lo)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float hx, lx, hy, ly, hz, lz;
    split_f64(src[4 * i], hx, lx);
    split_f64(src[4 * i + 1], hy, ly);
    split_f64(src[4 * i + 2], hz, lz);
    hi[i] = make_float4(hx, hy, hz, (float)src[4 * i + 3]);
    lo[i] = make_float4(lx, ly, lz, 0.f);
}

__global__ void split_targets_kernel(long long n, const double *tgt, float4 *hi, float4 *lo, double4_32a *t64)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = tgt[3 * i], y = tgt[3 * i + 1], z = tgt[3 * i + 2];
    t64[i] = make_double4_32a(x, y, z, 0.0);
    float hx, lx, hy, ly, hz, lz;
    split_f64(x, hx, lx);
    split_f64(y, hy, ly);
    split_f64(z, hz, lz);
    hi[i] = make_float4(hx, hy, hz, 0.f);
    lo[i] = make_float4(lx, ly, lz, 0.f);
}

__global__ void scatter_results_kernel(long long n, const double *phi, const double *e, double *pot, double *field)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    pot[i] = phi[i];
    if (field) {
        field[3 * i] = e[3 * i];
        field[3 * i + 1] = e[3 * i + 1];
        field[3 * i + 2] = e[3 * i + 2];
    }
}
}  // namespace

int hsma_coulomb_sum(int64_t ns, const double *src, int64_t nt, const double *tgt, double *pot, double *field,
                     int precision, void *stream)
{
    if (ns < 1 || nt < 1 || !src || !tgt || !pot) return HSMA_E_ARG;
    if (precision != HSMA_FP64 && precision != HSMA_FP32_ACC64) return HSMA_E_ARG;
    if (ns > (1LL << 31) || nt > (1LL << 30)) return HSMA_E_ARG;
    if (((uintptr_t)src | (uintptr_t)tgt | (uintptr_t)pot | (uintptr_t)field) & 7) return HSMA_E_ARG;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    HSMA_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    const int TB = pair_targets_per_block(precision);
    const int tile = precision == HSMA_FP64 ? 256 : 512;
    const int ctas = pair_max_ctas_per_sm(precision);
    const int slots = prop.multiProcessorCount * ctas;
    SysDesc d{};
    d.n = 0;
    d.ntb_part = 0;
    d.ntb = (int)((nt + TB - 1) / TB);
    double chunk = std::max(4.0 * tile, (double)d.ntb * ns / (24.0 * slots));
    long long maxchunks = std::max(1LL, (long long)((ns + tile - 1) / tile));
    d.nchunks = (int)std::max(1LL, std::min(maxchunks, (long long)llround(ns / chunk)));
    long long items = (long long)d.ntb * d.nchunks;
    if (items > (1LL << 30)) return HSMA_E_ARG;
    // sizes
    size_t bytes = 0;
    {
        Carver cc(nullptr);
        cc.take<float4>(ns);
        cc.take<float4>(ns);
        cc.take<double4_32a>(ns);
        cc.take<float4>(nt);
        cc.take<float4>(nt);
        cc.take<double4_32a>(nt);
        cc.take<float4>(2 * (size_t)d.nchunks * nt);
        cc.take<double>(nt);
        cc.take<double>(3 * nt);
        cc.take<long long>(1);
        cc.take<int>(8);
        cc.take<int>(1);
        cc.take<SysDesc>(1);
        bytes = align_up(cc.off, 256);
    }
    void *mem = nullptr;
    HSMA_CUDA_TRY(dev_malloc(&mem, bytes));
    Carver cc(mem);
    float4 *shi = cc.take<float4>(ns);
    float4 *slo = cc.take<float4>(ns);
    double4_32a *s64 = cc.take<double4_32a>(ns);
    float4 *thi = cc.take<float4>(nt);
    float4 *tlo = cc.take<float4>(nt);
    double4_32a *t64 = cc.take<double4_32a>(nt);
    float4 *partials = cc.take<float4>(2 * (size_t)d.nchunks * nt);
    double *phi = cc.take<double>(nt);
    double *e = cc.take<double>(3 * nt);
    long long *dns = cc.take<long long>(1);
    int *ctrl = cc.take<int>(8);
    int *status = cc.take<int>(1);
    SysDesc *dsys = cc.take<SysDesc>(1);
    int rc = HSMA_OK;
    long long nsl = ns;
    do {
        if (cudaMemcpyAsync(dsys, &d, sizeof(d), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(dns, &nsl, sizeof(nsl), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(ctrl, 0, 8 * sizeof(int), st) != cudaSuccess ||
            cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) {
            rc = HSMA_E_CUDA;
            break;
        }
        if (precision == HSMA_FP64 &&
            cudaMemcpyAsync(s64, src, sizeof(double) * 4 * ns, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
            rc = HSMA_E_CUDA;
            break;
        }
        if (precision != HSMA_FP64) {
            split_sources_kernel<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(ns, src, shi, slo);
            HSMA_LAUNCHED();
        }
        split_targets_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(nt, tgt, thi, tlo, t64);
        HSMA_LAUNCHED();
        PairArgs pa;
        pa.sys = dsys;
        pa.nsys = 1;
        pa.total_items = (int)items;
        pa.ns = dns;
        pa.src_hi = shi;
        pa.src_lo = slo;
        pa.src64 = s64;
        pa.ext_hi = thi;
        pa.ext_lo = tlo;
        pa.ext64 = t64;
        pa.n_ext = (int)nt;
        pa.ext_field = field ? 1 : 0;
        pa.ext_skip_zero = 1;
        pa.partials = partials;
        pa.next_item = ctrl;
        pa.status = status;
        int grid = (int)std::max(1LL, std::min(items, (long long)slots));
        if ((rc = launch_pair(pa, precision, 4, grid, st))) break;
        if ((rc = launch_partial_reduce(dsys, 1, nt, (int)nt, partials, precision, phi, e, st))) break;
        scatter_results_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(nt, phi, e, pot, field);
        HSMA_LAUNCHED();
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = HSMA_E_CUDA;
        int hst = 0;
        if (!rc && cudaMemcpy(&hst, status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = HSMA_E_CUDA;
        if (!rc) rc = map_status(hst);
    } while (0);
    dev_free(mem);
    if (rc == HSMA_OK && cudaGetLastError() != cudaSuccess) rc = HSMA_E_CUDA;
    return rc;
}

int hsma_basis(int p, double Rs, int64_t np, const double *pts, double *out, int precision, void *stream)
{
    if (p < 0 || p > 40 || !(Rs > 0) || np < 1 || !pts || !out) return HSMA_E_ARG;
    if (precision != HSMA_FP64 && precision != HSMA_FP32_ACC64) return HSMA_E_ARG;
    const int Nb = (p + 1) * (p + 1);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = precision == HSMA_FP32_ACC64 ? launch_basis_df(p, Rs, np, pts, 3, out, Nb, st)
                                          : launch_basis(p, Rs, np, pts, 3, out, Nb, st);
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = HSMA_E_CUDA;
    return rc;
}

}  // extern "C"
