// hsma_coulomb_sum_static: the direct Coulomb sum of hsma_coulomb_sum, for
// callers that must not allocate device memory at call time.
//
// Some callers cannot let a library call cudaMalloc/cudaFree while they run:
// a host application whose memory manager owns the whole device and forbids
// outside allocations after start-up, or a time-critical loop for which the
// implicit device-wide synchronisation of cudaFree is unacceptable.  This
// entry point takes all of its working memory from one array of
// kStaticScratchBytes that lives in this file as a static __device__ object:
// the driver reserves it when it loads this part of the library, every GPU
// that loads it keeps it until the process exits, and no call allocates.
//
// The array is shared by every call on a device and keeps the contents the
// last call left; each call first clears what must start at zero (work
// counter, status word) with a kernel.  Calls whose device work overlaps --
// on two streams, or from two host threads -- race on the array and give
// wrong results: serialise them.
//
// The first call on each device looks up the array's device address with
// cudaGetSymbolAddress (host code cannot use the symbol itself as a device
// pointer) and caches it with the identity of the current context; make that
// first call before any stream capture.  A later call in a different context
// (the device was reset, and the module loaded again) looks it up anew.
#include <cuda.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace hsma {

namespace {

constexpr size_t kStaticScratchBytes = (size_t)HSMA_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context id the address belongs to
int g_num_sms[kMaxDevices] = {};

// Process-unique id of the current context (cuCtxGetId), reached through the
// runtime's driver entry-point table so that the library needs no link
// against the driver library.  Returns false where the driver lacks it.
bool current_context_id(unsigned long long *id)
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    CUcontext c = nullptr;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct StaticLayout {
    size_t shi, slo, s64, thi, tlo, t64, partials, phi, e, ns, ctrl, status, sys, end;
};

// Byte offsets of every buffer inside the static array for one call.
StaticLayout layout_for(long long ns, long long nt, int nchunks, int precision)
{
    StaticLayout L;
    size_t o = 0;
    auto put = [&](size_t bytes) {
        size_t at = o;
        o = up256(o + bytes);
        return at;
    };
    const bool f64 = precision == HSMA_FP64;
    L.shi = put(f64 ? 0 : (size_t)ns * sizeof(float4));
    L.slo = put(f64 ? 0 : (size_t)ns * sizeof(float4));
    L.s64 = put(f64 ? (size_t)ns * sizeof(double4_32a) : 0);
    L.thi = put((size_t)nt * sizeof(float4));
    L.tlo = put((size_t)nt * sizeof(float4));
    L.t64 = put((size_t)nt * sizeof(double4_32a));
    L.partials = put((size_t)nchunks * nt * 2 * sizeof(float4));
    L.phi = put((size_t)nt * sizeof(double));
    L.e = put((size_t)nt * 3 * sizeof(double));
    L.ns = put(sizeof(long long));
    L.ctrl = put(8 * sizeof(int));
    L.status = put(sizeof(int));
    L.sys = put(sizeof(SysDesc));
    L.end = o;
    return L;
}

// Writes the work description and clears the counters and status.
__global__ void static_init_kernel(SysDesc d, long long ns, SysDesc *dsys, long long *dns, int *ctrl, int *status)
{
    if (threadIdx.x == 0) {
        *dsys = d;
        *dns = ns;
        *status = 0;
    }
    if (threadIdx.x < 8) ctrl[threadIdx.x] = 0;
}

__global__ void static_split_sources_kernel(long long n, const double *src, float4 *hi, float4 *lo,
                                            double4_32a *s64)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = src[4 * i], y = src[4 * i + 1], z = src[4 * i + 2], q = src[4 * i + 3];
    if (s64) {
        s64[i] = make_double4_32a(x, y, z, q);
        return;
    }
    float hx, lx, hy, ly, hz, lz;
    split_f64(x, hx, lx);
    split_f64(y, hy, ly);
    split_f64(z, hz, lz);
    hi[i] = make_float4(hx, hy, hz, (float)q);
    lo[i] = make_float4(lx, ly, lz, 0.f);
}

__global__ void static_split_targets_kernel(long long n, const double *tgt, float4 *hi, float4 *lo, double4_32a *t64)
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

__global__ void static_scatter_kernel(long long n, const double *phi, const double *e, double *pot, double *field)
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

// Once per device and context: the static array's device address and the
// SM count, looked up with the device current (the lookup itself makes the
// runtime's context current on a first call).  Without a context id from the
// driver, the address is looked up on every call.
int static_setup(int dev, void **addr, int *sms)
{
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (dev < 0 || dev >= kMaxDevices) return HSMA_E_ARG;
    unsigned long long ctx = 0;
    bool have_ctx = current_context_id(&ctx);
    if (!g_scratch_addr[dev] || !have_ctx || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        HSMA_CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
        int n = 0;
        HSMA_CUDA_TRY(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        have_ctx = current_context_id(&ctx);
        g_num_sms[dev] = n;
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = have_ctx ? ctx : 0;
    }
    *addr = g_scratch_addr[dev];
    *sms = g_num_sms[dev];
    return HSMA_OK;
}

}  // namespace

}  // namespace hsma

using namespace hsma;

extern "C" int hsma_coulomb_sum_static(int64_t ns, const double *src, int64_t nt, const double *tgt, double *pot,
                                       double *field, int precision, void *stream)
{
    if (ns < 1 || nt < 1 || !src || !tgt || !pot) return HSMA_E_ARG;
    if (precision != HSMA_FP64 && precision != HSMA_FP32_ACC64) return HSMA_E_ARG;
    if (((uintptr_t)src | (uintptr_t)tgt | (uintptr_t)pot | (uintptr_t)field) & 7) return HSMA_E_ARG;
    if (ns > (1LL << 31) || nt > (1LL << 30)) return HSMA_E_CAPACITY;
    int dev = 0;
    HSMA_CUDA_TRY(cudaGetDevice(&dev));
    void *base = nullptr;
    int sms = 0;
    int rc = static_setup(dev, &base, &sms);
    if (rc) return rc;

    // work decomposition as in hsma_coulomb_sum, with the chunk count lowered
    // until the call fits in the static array
    const int TB = pair_targets_per_block(precision);
    const int tile = precision == HSMA_FP64 ? 256 : 512;
    const int slots = sms * pair_max_ctas_per_sm(precision);
    SysDesc d{};
    d.n = 0;
    d.ntb_part = 0;
    d.ntb = (int)((nt + TB - 1) / TB);
    double chunk = std::max(4.0 * tile, (double)d.ntb * ns / (24.0 * slots));
    long long maxchunks = std::max(1LL, (long long)((ns + tile - 1) / tile));
    int nchunks = (int)std::max(1LL, std::min(maxchunks, (long long)llround(ns / chunk)));
    while (nchunks > 1 && layout_for(ns, nt, nchunks, precision).end > kStaticScratchBytes) nchunks = nchunks / 2;
    StaticLayout L = layout_for(ns, nt, nchunks, precision);
    if (L.end > kStaticScratchBytes) return HSMA_E_CAPACITY;
    d.nchunks = nchunks;
    const long long items = (long long)d.ntb * d.nchunks;
    if (items > (1LL << 30)) return HSMA_E_CAPACITY;

    char *b = (char *)base;
    float4 *shi = (float4 *)(b + L.shi), *slo = (float4 *)(b + L.slo);
    double4_32a *s64 = (double4_32a *)(b + L.s64);
    float4 *thi = (float4 *)(b + L.thi), *tlo = (float4 *)(b + L.tlo);
    double4_32a *t64 = (double4_32a *)(b + L.t64);
    float4 *partials = (float4 *)(b + L.partials);
    double *phi = (double *)(b + L.phi), *e = (double *)(b + L.e);
    long long *dns = (long long *)(b + L.ns);
    int *ctrl = (int *)(b + L.ctrl), *status = (int *)(b + L.status);
    SysDesc *dsys = (SysDesc *)(b + L.sys);
    cudaStream_t st = (cudaStream_t)stream;

    static_init_kernel<<<1, 32, 0, st>>>(d, ns, dsys, dns, ctrl, status);
    HSMA_LAUNCHED();
    const bool f64 = precision == HSMA_FP64;
    static_split_sources_kernel<<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(ns, src, f64 ? nullptr : shi,
                                                                              f64 ? nullptr : slo,
                                                                              f64 ? s64 : nullptr);
    HSMA_LAUNCHED();
    static_split_targets_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(nt, tgt, thi, tlo, t64);
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
    const int grid = (int)std::max(1LL, std::min(items, (long long)slots));
    if ((rc = launch_pair(pa, precision, 4, grid, st))) return rc;
    if ((rc = launch_partial_reduce(dsys, 1, nt, (int)nt, partials, precision, phi, e, st))) return rc;
    static_scatter_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(nt, phi, e, pot, field);
    HSMA_LAUNCHED();
    HSMA_CUDA_TRY(cudaGetLastError());
    int hst = 0;
    HSMA_CUDA_TRY(cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    HSMA_CUDA_TRY(cudaStreamSynchronize(st));
    if (hst & ST_TIMEOUT) return HSMA_E_TIMEOUT;
    return HSMA_OK;
}
