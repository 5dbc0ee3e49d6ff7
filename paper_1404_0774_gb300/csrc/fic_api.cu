// Host side of the C ABI declared in include/fic.h.
//
// fic_encode runs, on one stream: (host image -> device copy) -> prep
// (ranges, domain pool) -> search (tensor-core or SIMT screening) -> exact
// re-score + certification -> exact fallback for uncertified ranges ->
// final FP64 codes and residuals -> (device -> host maps copy).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fic_internal.cuh"

using namespace fic;

namespace {

thread_local int64_t g_stats[4] = {0, 0, 0, 0};

// Phase events of the last timed encode (per host thread).
struct PhaseEvents {
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool valid = false;
    bool ensure()
    {
        for (auto &e : ev)
            if (!e && cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
        return true;
    }
};
thread_local PhaseEvents g_phase;

// Events around the search of each quadtree level (fic_encode_quadtree with
// FIC_FLAG_PHASE_TIMING).
struct QtPhaseEvents {
    cudaEvent_t ev[kMaxLevels][2] = {};
    int levels = 0;
    bool valid = false;
    bool ensure()
    {
        for (auto &l : ev)
            for (auto &e : l)
                if (!e && cudaEventCreate(&e) != cudaSuccess) {
                    cudaGetLastError();
                    return false;
                }
        return true;
    }
};
thread_local QtPhaseEvents g_qt_phase;

constexpr size_t kAlign = 256;
size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

int check_params(const fic_params *p)
{
    if (!p) return FIC_ERR_BAD_ARG;
    if (p->flags & ~(FIC_FLAG_PHASE_TIMING | FIC_FLAG_DENSE | FIC_FLAG_EXACT_SCAN)) return FIC_ERR_BAD_ARG;
    if (p->range_size != 4 && p->range_size != 8 && p->range_size != 16) return FIC_ERR_BAD_ARG;
    if (p->domain_stride < 1) return FIC_ERR_BAD_ARG;
    if (p->bit_depth < 1 || p->bit_depth > 12) return FIC_ERR_BITDEPTH;
    if (p->s_bits < 2 || p->s_bits > 8 || p->o_bits < 2 || p->o_bits > 10) return FIC_ERR_BITDEPTH;
    if (p->decode_iters < 0 || p->decode_iters > 100000) return FIC_ERR_BAD_ARG;
    if (p->search < FIC_SEARCH_AUTO || p->search > FIC_SEARCH_SIMT) return FIC_ERR_BAD_ARG;
    if (p->n_split < 0) return FIC_ERR_BAD_ARG;
    return FIC_OK;
}

int make_geometry(int w, int h, int pitch, const fic_params *p, Geometry &g)
{
    int rc = check_params(p);
    if (rc != FIC_OK) return rc;
    const int n = p->range_size;
    if (w <= 0 || h <= 0 || w % n || h % n || w < 2 * n || h < 2 * n) return FIC_ERR_SIZE;
    if (pitch < w) return FIC_ERR_BAD_ARG;
    if ((long long)w * h > (1LL << 30)) return FIC_ERR_SIZE;
    std::memset(&g, 0, sizeof g);
    g.w = w;
    g.h = h;
    g.pitch = pitch;
    g.n = n;
    g.t = p->domain_stride;
    g.m = n * n;
    g.ln = n == 4 ? 2 : (n == 8 ? 3 : 4);
    g.nx = w / n;
    g.ny = h / n;
    g.R = g.nx * g.ny;
    g.U = (w - 2 * n) / g.t + 1;
    g.V = (h - 2 * n) / g.t + 1;
    if ((long long)g.U * g.V * 8 >= (1LL << 31)) return FIC_ERR_SIZE;
    g.D = g.U * g.V;
    g.N = 8 * g.D;
    g.B = p->bit_depth;
    g.P = (1 << g.B) - 1;
    g.s_bits = p->s_bits;
    g.o_bits = p->o_bits;
    g.Ls = (1 << (g.s_bits - 1)) - 1;
    g.Lo = (1 << (g.o_bits - 1)) - 1;
    g.split_hilo = 4 * g.P > 2048 ? 1 : 0;
    g.KP = (g.split_hilo ? 2 * g.m : g.m) + 16;
    const long long Gnum = 4LL * g.Ls * g.m * g.P;
    g.mod_g = (Gnum % g.Lo) == 0 ? 1 : 0;
    g.G = (double)Gnum / g.Lo;
    g.Gi = g.mod_g ? (int)(Gnum / g.Lo) : 0;
    {
        // magnitude of the exact residual expansion R*D^2 (sum of the absolute
        // values of its six terms at the largest statistics this bit depth
        // allows): 64-bit integers suffice below 2^62
        const double m = g.m, P = g.P, Ls = g.Ls, Lo = g.Lo;
        const double A = Ls * Lo, Bo = 4.0 * Ls * Lo * P, Dd = 4.0 * Ls * Lo;
        const double Sq = m * 4.0 * P, Sqq = m * 16.0 * P * P, Sb = m * P, Sbb = m * P * P, X = m * 4.0 * P * P;
        const double bound = A * A * Sqq + m * Bo * Bo + Dd * Dd * Sbb + 2.0 * A * Bo * Sq + 2.0 * A * Dd * X +
                             2.0 * Bo * Dd * Sb;
        g.wide = bound < 4.0e18 ? 0 : 1;  // 2^62 = 4.61e18
    }
    return FIC_OK;
}

EpiConst make_epi(const Geometry &g)
{
    EpiConst ec;
    ec.two_ls = 2.0f * g.Ls;
    ec.ls = (float)g.Ls;
    ec.inv2ls = (float)(0.5 / g.Ls);
    ec.G = (float)g.G;
    ec.invG = (float)(1.0 / g.G);
    const double pl = (double)g.P / g.Lo;
    const double lambda = 2.0 * g.Ls * g.m * pl * pl / (g.G * g.G);
    ec.lambda = (float)lambda;
    ec.delta_o = (float)(g.m * 0.25 * pl * pl);
    // o code decided next to its rounding boundary: z/G is off by at most
    // eps (z units) -> the residue w moves by eps and lambda*w^2 by
    // lambda*(G*eps + eps^2) around |w| = G/2; eps covers the FP32 rounding of
    // z*invG and of the residue (z spans up to 16*G when reduced mod G, else
    // 8*Ls*m*P)
    const double zmax = g.mod_g ? 16.0 * g.G : 8.0 * g.Ls * g.m * g.P;
    const double eps = zmax * 2.384185791015625e-07 + (g.mod_g ? 0.0 : g.Lo * g.G * 1.2e-7);  // 2^-22
    ec.beta_o = (float)(2.0 * lambda * (g.G * eps + eps * eps) + 1e-3);
    ec.sqrtm4 = (float)(0.25 * sqrt((double)g.m));
    ec.inv4ls = (float)(0.25 / g.Ls);
    ec.invm = (float)(1.0 / g.m);
    ec.pmax = (float)g.P - 0.5f;
    ec.near_slack = (float)((32.0 * g.Ls * g.Ls + 16.0 * g.Ls) * 5.9604644775390625e-08);  // 2^-24
    const double dd = 4.0 * g.Ls * g.Lo;
    ec.invD2_up = std::nextafter((float)(1.0 / (dd * dd)), INFINITY);
    // the residue w = z - round(z/G) G of the FP32 key: |w| <= G/2 plus the
    // rounding of z*invG (2^-23 |z|, taken as 2^-22 zmax), lambda w^2 then
    // rounded once more
    const double wmax = 0.5 * g.G + zmax * 2.384185791015625e-07;
    ec.qmax = (float)(lambda * wmax * wmax * 1.001 + 1.0);
    return ec;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
    return n > 0 ? n : 148;
}

int choose_search(const Geometry &g, const fic_params *p)
{
    if (p->search == FIC_SEARCH_SIMT) return FIC_SEARCH_SIMT;
    if (search_tc_supported(g)) return FIC_SEARCH_TC;
    return p->search == FIC_SEARCH_TC ? -1 : FIC_SEARCH_SIMT;
}

// Maximum split of the candidate dimension (the list layout).  The kernels
// use fewer splits when fewer ranges and domains need screening: enough work
// for `target` (three work items per SM for the persistent tensor-core search,
// measured a little faster than two or four on the 512x512 slice; eight CTAs
// per SM for the FP32 search), see active_splits.
constexpr int kMaxSplit = 64;
constexpr int kMaxLists = 128;  // candidate lists per range the re-score takes (and its work-item codes hold)

int lists_per_split(int search);

int choose_split(const Geometry &g, const fic_params *p, int search)
{
    (void)g;
    const int cap = std::min(kMaxSplit, kMaxLists / lists_per_split(search));
    return p->n_split > 0 ? std::min(p->n_split, cap) : cap;
}

int split_target(const fic_params *p, int search)
{
    if (p->n_split > 0) return 1 << 30;  // a fixed split: active_splits caps it at max_split
    return (search == FIC_SEARCH_TC ? 3 : 8) * sm_count();
}

// How the search forms the cross term, for the statistics' error allowances:
// 0 with the FP32 search or the exact 8-bit tensor-core layout (centring in
// the MMA), 1 with exact hi/lo tensor-core accumulators (12-bit, K <= 64), 2
// with tensor-core accumulation over K = 256 per part (16x16 ranges); 1 and 2
// fold the centring correction into the epilogue.
int tc_mode_of(const Geometry &g, int search)
{
    if (search != FIC_SEARCH_TC) return 0;
    if (g.m == 256) return 2;
    return g.split_hilo ? 1 : 0;
}

int lists_per_split(int search)
{
    return search == FIC_SEARCH_SIMT ? search_simt_lists_per_split() : search_tc_lists_per_split();
}

struct EncLayout {
    size_t img, ri, di, dconst, bblk, qblk, rs32, cb32, ra16, cb16, lists, winner, winx, fb_list, fb_count, span,
        tbest, partial, maps, rkeep, dkeep, act, dact, counts, dconst_c, dmap, bmask, bcount, total;
};

// tc_operands = false: the tensor-core operand rows live elsewhere (a
// batch keeps every slice's in one shared pair of buffers).
EncLayout enc_layout(const Geometry &g, int search, int n_lists, bool tc_operands = true)
{
    EncLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const size_t elem = g.B <= 8 ? 1 : 2;
    L.img = take((size_t)g.w * g.h * elem);
    L.ri = take(sizeof(RangeInfo) * g.R);
    L.di = take(sizeof(DomainInfo) * g.D);
    L.dconst = take(sizeof(float4) * g.D);
    L.bblk = take(sizeof(uint16_t) * (size_t)g.R * g.m);
    L.qblk = take(sizeof(uint16_t) * (size_t)g.D * g.m);
    const bool simt = search == FIC_SEARCH_SIMT;
    L.rs32 = simt ? take(sizeof(float) * (size_t)g.R * g.m) : 0;
    L.cb32 = simt ? take(sizeof(float) * (size_t)g.N * g.m) : 0;
    L.ra16 = simt || !tc_operands ? 0 : take(sizeof(__half) * (size_t)search_tc_rows(g.R) * g.KP);
    L.cb16 = simt || !tc_operands ? 0 : take(sizeof(__half) * (size_t)search_tc_cols(g.N) * g.KP);
    L.lists = take(sizeof(ListEntry) * (size_t)g.R * n_lists * kListK);
    L.winner = take(sizeof(uint32_t) * g.R);
    L.winx = take(sizeof(long long) * g.R);
    L.fb_list = take(sizeof(int) * g.R);
    L.fb_count = take(sizeof(int) * 4);  // full-scan count, error flag, list-scan count, search work items
    L.span = take(span_bytes(g, n_lists));
    L.tbest = take(sizeof(int) * g.R);
    L.partial = take(fallback_partial_bytes(g));
    L.maps = take(sizeof(fic_map) * g.R);
    L.rkeep = take(sizeof(int) * g.R);
    L.dkeep = take(sizeof(int) * g.D);
    L.act = take(sizeof(int) * g.R);
    L.dact = take(sizeof(int) * g.D);
    L.counts = take(sizeof(int) * 4);
    L.dconst_c = take(sizeof(float4) * g.D);
    L.dmap = take(sizeof(int) * g.D);
    L.bmask = take(sizeof(uint4) * stats_grid(g));
    L.bcount = take(sizeof(int) * stats_grid(g));
    L.total = o;
    return L;
}

bool is_device_ptr(const void *ptr)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Where a caller's buffer lives: device (or managed) memory, page-locked host
// memory that kernels can address (its device address in *dev), or other
// host memory, which only the copy engines reach.
enum class Mem { Device, PinnedHost, Host };

Mem classify(const void *ptr, void **dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return Mem::Host;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return Mem::Device;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *dev = a.devicePointer;
        return Mem::PinnedHost;
    }
    return Mem::Host;
}

// The image from page-locked host memory into the workspace, 16 bytes a
// thread: for half a megabyte a kernel over the chip-to-chip link costs a
// few microseconds, a copy-engine transfer about twelve (most of it the
// operation's fixed latency).  The loads go first, the stores after the wait
// for the stream's previous kernel.
__global__ void __launch_bounds__(256) k_copy_in(const uint4 *__restrict__ src, uint4 *__restrict__ dst, size_t n16)
{
    const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, step = (size_t)gridDim.x * blockDim.x;
    uint4 v[4];
    int k = 0;
    for (size_t i = i0; i < n16 && k < 4; i += step, ++k) v[k] = __ldcs(src + i);
    grid_dep_sync();
    k = 0;
    for (size_t i = i0; i < n16 && k < 4; i += step, ++k) dst[i] = v[k];
    for (size_t i = i0 + 4 * step; i < n16; i += step) dst[i] = __ldcs(src + i);
}

// A pinned host word of this thread for reading the device error flag back
// after a call with host buffers (allocated on the thread's first such call
// and kept; a pageable destination would route the 4-byte copy through a
// staging buffer).  Null when it cannot be had or when the caller may not
// allocate (fic_encode_static): the copy then goes to a stack word.
thread_local bool g_no_alloc = false;

int *pinned_flag()
{
    thread_local int *flag = nullptr;
    thread_local bool tried = false;
    if (!flag && !tried && !g_no_alloc) {
        tried = true;
        if (cudaMallocHost(reinterpret_cast<void **>(&flag), sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            flag = nullptr;
        }
    }
    return g_no_alloc ? nullptr : flag;
}

// Pinned host words of this thread for reading n ints back (as pinned_flag;
// null when they cannot be had).
int *pinned_words(int n)
{
    thread_local int *buf = nullptr;
    thread_local int have = 0, failed_at = 0;  // failed_at: a request of this size could not be met
    if (have < n && !g_no_alloc && (failed_at == 0 || n < failed_at)) {
        if (buf) cudaFreeHost(buf);
        buf = nullptr;
        have = 0;
        if (cudaMallocHost(reinterpret_cast<void **>(&buf), sizeof(int) * n) == cudaSuccess) {
            have = n;
        } else {
            cudaGetLastError();
            buf = nullptr;
            failed_at = n;
        }
    }
    return have >= n ? buf : nullptr;
}

// FIC_DEBUG=1 in the environment: synchronise after every call on the
// encode/decode paths and report the first failing one on stderr.
bool debug_mode()
{
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FIC_DEBUG");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v == 1;
}

cudaError_t debug_check(cudaError_t e, const char *what, int line, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (e == cudaSuccess && debug_mode() && cudaStreamIsCapturing(st, &cs) == cudaSuccess &&
        cs == cudaStreamCaptureStatusNone)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && debug_mode())
        fprintf(stderr, "libfic: %s failed at fic_api.cu:%d: %s\n", what, line, cudaGetErrorString(e));
    return e;
}

#define FIC_CUDA(call)                                              \
    do {                                                            \
        cudaError_t e_ = debug_check((call), #call, __LINE__, st);  \
        if (e_ != cudaSuccess) {                                    \
            cudaGetLastError();                                     \
            rc = FIC_ERR_CUDA;                                      \
            goto done;                                              \
        }                                                           \
    } while (0)

}  // namespace

extern "C" {

void fic_default_params(fic_params *p)
{
    if (!p) return;
    p->range_size = 8;
    p->domain_stride = 8;
    p->bit_depth = 8;
    p->s_bits = 5;
    p->o_bits = 7;
    p->decode_iters = 10;
    p->search = FIC_SEARCH_AUTO;
    p->n_split = 0;
    p->flags = 0;
}

int fic_counts(int w, int h, const fic_params *p, int64_t *n_ranges, int64_t *n_domains)
{
    Geometry g;
    const int rc = make_geometry(w, h, w, p, g);
    if (rc != FIC_OK) return rc;
    if (n_ranges) *n_ranges = g.R;
    if (n_domains) *n_domains = g.D;
    return FIC_OK;
}

int fic_encode_workspace_size(int w, int h, const fic_params *p, size_t *bytes)
{
    if (!bytes) return FIC_ERR_BAD_ARG;
    Geometry g;
    const int rc = make_geometry(w, h, w, p, g);
    if (rc != FIC_OK) return rc;
    const int search = choose_search(g, p);
    if (search < 0) return FIC_ERR_UNSUPPORTED;
    *bytes = enc_layout(g, search, choose_split(g, p, search) * lists_per_split(search)).total;
    return FIC_OK;
}

}  // extern "C"

namespace {


EncBufs enc_bufs(const EncLayout &L, char *ws)
{
    EncBufs b;
    b.ri = reinterpret_cast<RangeInfo *>(ws + L.ri);
    b.di = reinterpret_cast<DomainInfo *>(ws + L.di);
    b.dconst = reinterpret_cast<float4 *>(ws + L.dconst);
    b.bblk = reinterpret_cast<uint16_t *>(ws + L.bblk);
    b.qblk = reinterpret_cast<uint16_t *>(ws + L.qblk);
    b.rs32 = L.rs32 ? reinterpret_cast<float *>(ws + L.rs32) : nullptr;
    b.cb32 = L.cb32 ? reinterpret_cast<float *>(ws + L.cb32) : nullptr;
    b.ra16 = L.ra16 ? reinterpret_cast<__half *>(ws + L.ra16) : nullptr;
    b.cb16 = L.cb16 ? reinterpret_cast<__half *>(ws + L.cb16) : nullptr;
    b.lists = reinterpret_cast<ListEntry *>(ws + L.lists);
    b.winner = reinterpret_cast<uint32_t *>(ws + L.winner);
    b.winx = reinterpret_cast<long long *>(ws + L.winx);
    b.fb_list = reinterpret_cast<int *>(ws + L.fb_list);
    b.fb_count = reinterpret_cast<int *>(ws + L.fb_count);
    b.err = b.fb_count + 1;
    b.tbest = reinterpret_cast<int *>(ws + L.tbest);
    b.partial = ws + L.partial;
    b.span = ws + L.span;
    b.cb.rkeep = reinterpret_cast<int *>(ws + L.rkeep);
    b.cb.dkeep = reinterpret_cast<int *>(ws + L.dkeep);
    b.cb.act = reinterpret_cast<int *>(ws + L.act);
    b.cb.dact = reinterpret_cast<int *>(ws + L.dact);
    b.cb.counts = reinterpret_cast<int *>(ws + L.counts);
    b.cb.dconst_c = reinterpret_cast<float4 *>(ws + L.dconst_c);
    b.cb.dmap = reinterpret_cast<int *>(ws + L.dmap);
    b.cb.bmask = reinterpret_cast<uint4 *>(ws + L.bmask);
    b.cb.bcount = reinterpret_cast<int *>(ws + L.bcount);
    return b;
}

// The device pipeline of one encode on a prepared workspace (no allocation,
// no synchronisation): statistics, compaction, operand rows, seed, search,
// re-score, exact fallback, map output.  dimg: device image with row pitch
// gd.pitch; active (nullable): only ranges with active[r] != 0 are screened
// (the maps of the others are placeholders); dump != nullptr: stop after the
// contraction and write the raw cross terms there.
cudaError_t encode_pipeline(const Geometry &gd, const fic_params *p, int search, int n_split, int target,
                            const EncLayout &L, char *ws, const void *dimg, const int *active, fic_map *dmaps,
                            float *dump, bool timed, cudaStream_t st, const cudaEvent_t *search_ev = nullptr)
{
    const EncBufs b = enc_bufs(L, ws);
    const int n_lists = n_split * lists_per_split(search);
    // the contraction dump covers every range and candidate
    const int dense = (dump || (p->flags & FIC_FLAG_DENSE)) ? 1 : 0;
    const EpiConst ec = make_epi(gd);
    cudaError_t e;
#define FIC_STEP(call)                                                 \
    do {                                                               \
        if ((e = debug_check((call), #call, __LINE__, st)) != cudaSuccess) \
            return e;                                                  \
    } while (0)
#define FIC_MARK(i) \
    if (timed) FIC_STEP(cudaEventRecord(g_phase.ev[i], st))
    // (operand rows past the kept ones, padding included, are never written:
    // whatever they hold only reaches accumulator rows and columns that the
    // epilogue ignores; the exact-scan queue counters are zeroed by k_stats)
    FIC_MARK(0);
    FIC_STEP(launch_prep(gd, dimg, ec, dense, tc_mode_of(gd, search), active, b.ri, b.di, b.dconst, b.bblk, b.qblk, b.rs32, b.cb32, b.ra16,
                         b.cb16, b.tbest, b.cb, b.fb_count, dump ? 0 : 1, st));
    FIC_MARK(1);
    if (search_ev) FIC_STEP(cudaEventRecord(search_ev[0], st));
    if (search == FIC_SEARCH_TC)
        FIC_STEP(launch_search_tc(gd, ec, b.ri, b.cb, dense, b.ra16, b.cb16, b.lists, n_split, target, b.tbest, dump,
                                  b.err, b.fb_count + 3, st));
    else
        FIC_STEP(launch_search_simt(gd, ec, b.ri, b.di, b.cb, dense, b.rs32, b.cb32, b.lists, n_split, target, b.tbest,
                                    dump, st));
    if (search_ev) FIC_STEP(cudaEventRecord(search_ev[1], st));
    FIC_MARK(2);
    if (!dump) {
        FIC_STEP(launch_rescore(gd, ec, b.ri, b.di, b.bblk, b.qblk, b.lists, n_lists, b.cb.counts, b.cb.act, b.cb.rkeep,
                                lists_per_split(search), search == FIC_SEARCH_TC ? search_tc_tile() : 64, target,
                                n_split, sm_count(), (p->flags & FIC_FLAG_EXACT_SCAN) ? 1 : 0, b.winner, b.winx, b.fb_list,
                                b.fb_count, b.partial, b.span, st));
        FIC_MARK(3);
        FIC_STEP(launch_scans_finalize(gd, b.ri, b.di, b.bblk, b.qblk, b.fb_list, b.fb_count, b.partial, b.cb.counts,
                                       b.cb.dmap, search == FIC_SEARCH_TC ? search_tc_tile() : 64, target, n_split,
                                       lists_per_split(search), n_lists, b.span, b.winner, b.winx, b.err, dmaps, ec,
                                       b.dconst, sm_count(), st));
        FIC_MARK(4);
        FIC_MARK(5);
    }
#undef FIC_MARK
#undef FIC_STEP
    return cudaSuccess;
}

// Shared front end of fic_encode and fic_cross_terms (dump != nullptr: stop
// after the contraction and write the raw cross terms there).
int run_encode(const void *img, int w, int h, int pitch_px, const fic_params *p, fic_map *maps, int maps_cap,
               int *n_maps, void *workspace, size_t workspace_bytes, void *stream, float *dump)
{
    if (!img || (!maps && !dump)) return FIC_ERR_BAD_ARG;
    Geometry g;
    int rc = make_geometry(w, h, pitch_px, p, g);
    if (rc != FIC_OK) return rc;
    if (!dump && maps_cap < g.R) return FIC_ERR_CAPACITY;
    const int search = choose_search(g, p);
    if (search < 0) return FIC_ERR_UNSUPPORTED;
    const int n_split = choose_split(g, p, search);
    const int n_lists = n_split * lists_per_split(search);
    const EncLayout L = enc_layout(g, search, n_lists);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    bool owned = false;
    if (ws) {
        if (workspace_bytes < L.total) return FIC_ERR_CAPACITY;
        if (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) return FIC_ERR_BAD_ARG;
    } else {
        if (cudaMallocAsync(reinterpret_cast<void **>(&ws), L.total, st) != cudaSuccess) {
            cudaGetLastError();
            return FIC_ERR_CUDA;
        }
        owned = true;
    }
    {
        void *img_alias = nullptr, *maps_alias = nullptr;
        const Mem img_mem = classify(img, &img_alias);
        const Mem maps_mem = dump ? Mem::Device : classify(maps, &maps_alias);
        const bool img_dev = img_mem == Mem::Device, maps_dev = maps_mem == Mem::Device;
        const size_t elem = g.B <= 8 ? 1 : 2;
        const void *dimg = img;
        Geometry gd = g;
        if (!img_dev) {
            const size_t bytes = (size_t)w * h * elem;
            if (img_mem == Mem::PinnedHost && pitch_px == w && bytes % 16 == 0 &&
                (reinterpret_cast<uintptr_t>(img_alias) & 15) == 0) {
                const size_t n16 = bytes / 16;
                const int blocks = (int)std::min<size_t>((n16 + 255) / 256, (size_t)4 * sm_count());
                FIC_CUDA(launch_dep(k_copy_in, dim3(blocks), dim3(256), 0, st, (const uint4 *)img_alias,
                                    reinterpret_cast<uint4 *>(ws + L.img), n16));
            } else if (pitch_px == w) {  // one contiguous copy
                FIC_CUDA(cudaMemcpyAsync(ws + L.img, img, bytes, cudaMemcpyHostToDevice, st));
            } else {
                FIC_CUDA(cudaMemcpy2DAsync(ws + L.img, (size_t)w * elem, img, (size_t)pitch_px * elem,
                                           (size_t)w * elem, h, cudaMemcpyHostToDevice, st));
            }
            dimg = ws + L.img;
            gd.pitch = w;
        }
        // maps in page-locked host memory are written there by the map output
        // kernel itself (no copy back); every map carries FIC_MAP_ERROR when
        // the search set the error word, so the host reads it from map 0
        const bool maps_direct = maps_mem == Mem::PinnedHost;
        fic_map *dmaps = maps_dev ? maps
                                  : (maps_direct ? static_cast<fic_map *>(maps_alias)
                                                 : reinterpret_cast<fic_map *>(ws + L.maps));
        const bool timed = !dump && (p->flags & FIC_FLAG_PHASE_TIMING) && g_phase.ensure();
        g_phase.valid = false;
        FIC_CUDA(encode_pipeline(gd, p, search, n_split, split_target(p, search), L, ws, dimg, nullptr, dmaps, dump,
                                 timed, st));
        g_phase.valid = timed;
        const bool sync = dump || !maps_dev || !img_dev || debug_mode();
        if (!dump && !maps_dev && !maps_direct)
            FIC_CUDA(cudaMemcpyAsync(maps, dmaps, sizeof(fic_map) * g.R, cudaMemcpyDeviceToHost, st));
        if (sync) {
            int herr_stack = 0;
            int *hf = maps_direct ? nullptr : pinned_flag();
            int *dst = hf ? hf : &herr_stack;
            if (!maps_direct)
                FIC_CUDA(cudaMemcpyAsync(dst, enc_bufs(L, ws).err, sizeof(int), cudaMemcpyDeviceToHost, st));
            FIC_CUDA(cudaStreamSynchronize(st));
            const int herr = maps_direct ? (int)((maps[0].info & FIC_MAP_ERROR) != 0) : *dst;
            if (herr) {
                rc = FIC_ERR_TIMEOUT;
                if (debug_mode()) fprintf(stderr, "libfic: device error flag %d\n", herr);
            }
        }
        g_stats[0] = -1;
        g_stats[1] = n_lists;
        g_stats[2] = search;
        g_stats[3] = n_split;
        if (n_maps) *n_maps = g.R;
    }
done:
    if (owned) {
        if (cudaFreeAsync(ws, st) != cudaSuccess) {
            cudaGetLastError();
            if (rc == FIC_OK) rc = FIC_ERR_CUDA;
        }
    }
    return rc;
}

// ------------------------------------------------------------ quadtree

thread_local int64_t g_qt_stats[1 + 4 * kMaxLevels] = {0};

// Launch shapes chosen by timing, per level geometry.
struct TuneKey {
    int w, h, n, B, sb, ob, flags, fixed_search;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(w, h, n, B, sb, ob, flags, fixed_search) <
               std::tie(o.w, o.h, o.n, o.B, o.sb, o.ob, o.flags, o.fixed_search);
    }
};
struct TuneChoice {
    int search, waves;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune;

constexpr int kWaveChoices[3] = {2, 4, 8};

int target_for(int search, int waves) { return waves * (search == FIC_SEARCH_TC ? 1 : 2) * sm_count(); }

struct QtPlan {
    int levels;
    fic_params pl[kMaxLevels];
    Geometry g[kMaxLevels];
    size_t img, enc, active[kMaxLevels + 1], leaf[kMaxLevels], maps[kMaxLevels], lists, stage, counts, total;
    size_t enc_bytes;
};

int qt_plan(int w, int h, int pitch, const fic_params *p, int min_size, int maps_cap_check, QtPlan &Q)
{
    if (!p) return FIC_ERR_BAD_ARG;
    int rc = check_params(p);
    if (rc != FIC_OK) return rc;
    const int nmax = p->range_size;
    if (nmax != 8 && nmax != 16) return FIC_ERR_BAD_ARG;
    if ((min_size != 4 && min_size != 8 && min_size != 16) || min_size > nmax) return FIC_ERR_BAD_ARG;
    Q.levels = nmax == min_size ? 1 : (nmax / min_size == 2 ? 2 : 3);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    Q.enc_bytes = 0;
    for (int l = 0; l < Q.levels; ++l) {
        Q.pl[l] = *p;
        Q.pl[l].flags &= ~FIC_FLAG_PHASE_TIMING;  // a level's own phases are not recorded
        Q.pl[l].range_size = nmax >> l;
        Q.pl[l].domain_stride = nmax >> l;
        rc = make_geometry(w, h, pitch, &Q.pl[l], Q.g[l]);
        if (rc != FIC_OK) return rc;
        for (int s = FIC_SEARCH_TC; s <= FIC_SEARCH_SIMT; ++s) {
            if (s == FIC_SEARCH_TC && !search_tc_supported(Q.g[l])) continue;
            if (p->search != FIC_SEARCH_AUTO && p->search != s && !(s == FIC_SEARCH_SIMT && !search_tc_supported(Q.g[l])))
                continue;
            Q.enc_bytes = std::max(Q.enc_bytes, enc_layout(Q.g[l], s, choose_split(Q.g[l], p, s) * lists_per_split(s)).total);
        }
    }
    (void)maps_cap_check;
    const size_t elem = Q.g[0].B <= 8 ? 1 : 2;
    Q.img = take((size_t)w * h * elem);
    Q.enc = take(Q.enc_bytes);
    for (int l = 0; l < Q.levels; ++l) {
        Q.active[l] = take(sizeof(int) * Q.g[l].R);
        Q.leaf[l] = take(sizeof(int) * Q.g[l].R);
        Q.maps[l] = take(sizeof(fic_map) * Q.g[l].R);
    }
    Q.active[Q.levels] = take(sizeof(int));  // the last level splits nothing
    const size_t max_leaves = (size_t)(w / min_size) * (h / min_size);
    size_t nlist = 0;
    for (int l = 0; l < Q.levels; ++l) nlist += Q.g[l].R;
    Q.lists = take(sizeof(int) * nlist);
    Q.stage = take(sizeof(fic_qmap) * max_leaves);
    Q.counts = take(sizeof(int) * (2 + 2 * kMaxLevels));
    Q.total = o;
    return FIC_OK;
}

// Time one full pipeline run (after one warm-up run) in milliseconds.
float time_pipeline(const Geometry &g, const fic_params *p, int search, int target, const EncLayout &L, char *ws,
                    const void *dimg, const int *active, fic_map *dmaps, cudaStream_t st)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return 1e30f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return 1e30f;
    }
    const int n_split = choose_split(g, p, search);
    float ms = 1e30f;
    if (encode_pipeline(g, p, search, n_split, target, L, ws, dimg, active, dmaps, nullptr, false, st) ==
            cudaSuccess &&
        cudaEventRecord(a, st) == cudaSuccess &&
        encode_pipeline(g, p, search, n_split, target, L, ws, dimg, active, dmaps, nullptr, false, st) ==
            cudaSuccess &&
        cudaEventRecord(b, st) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess)
        cudaEventElapsedTime(&ms, a, b);
    cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

int run_quadtree(const void *img, int w, int h, int pitch_px, const fic_params *p, int min_size, float rms_split,
                 fic_qmap *maps, int maps_cap, int *n_maps, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!img || !maps) return FIC_ERR_BAD_ARG;
    QtPlan Q;
    int rc = qt_plan(w, h, pitch_px, p, min_size, maps_cap, Q);
    if (rc != FIC_OK) return rc;
    if ((size_t)maps_cap < (size_t)(w / min_size) * (h / min_size)) return FIC_ERR_CAPACITY;
    if (!(rms_split >= 0.0f)) return FIC_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    bool owned = false;
    if (ws) {
        if (workspace_bytes < Q.total) return FIC_ERR_CAPACITY;
        if (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) return FIC_ERR_BAD_ARG;
    } else {
        if (cudaMallocAsync(reinterpret_cast<void **>(&ws), Q.total, st) != cudaSuccess) {
            cudaGetLastError();
            return FIC_ERR_CUDA;
        }
        owned = true;
    }
    {
        void *img_alias = nullptr, *maps_alias = nullptr;
        const Mem img_mem = classify(img, &img_alias), maps_mem = classify(maps, &maps_alias);
        const bool maps_dev = maps_mem == Mem::Device;
        const size_t elem = Q.g[0].B <= 8 ? 1 : 2;
        const void *dimg = img;
        int pitch = pitch_px;
        if (img_mem != Mem::Device) {
            const size_t bytes = (size_t)w * h * elem;
            if (img_mem == Mem::PinnedHost && pitch_px == w && bytes % 16 == 0 &&
                (reinterpret_cast<uintptr_t>(img_alias) & 15) == 0) {
                const size_t n16 = bytes / 16;
                const int blocks = (int)std::min<size_t>((n16 + 255) / 256, (size_t)4 * sm_count());
                FIC_CUDA(launch_dep(k_copy_in, dim3(blocks), dim3(256), 0, st, (const uint4 *)img_alias,
                                    reinterpret_cast<uint4 *>(ws + Q.img), n16));
            } else {
                FIC_CUDA(cudaMemcpy2DAsync(ws + Q.img, (size_t)w * elem, img, (size_t)pitch_px * elem,
                                           (size_t)w * elem, h, cudaMemcpyHostToDevice, st));
            }
            dimg = ws + Q.img;
            pitch = w;
        }
        int *counts = reinterpret_cast<int *>(ws + Q.counts);
        FIC_CUDA(cudaMemsetAsync(counts, 0, sizeof(int) * (2 + 2 * kMaxLevels), st));
        FIC_CUDA(cudaMemsetAsync(ws + Q.active[0], 1, sizeof(int) * Q.g[0].R, st));  // every level-0 range
        QtLevels lv;
        lv.levels = Q.levels;
        int list_off = 0;
        const bool timed = (p->flags & FIC_FLAG_PHASE_TIMING) && g_qt_phase.ensure();
        g_qt_phase.valid = false;
        g_qt_stats[0] = Q.levels;
        for (int l = 0; l < Q.levels; ++l) {
            Geometry g = Q.g[l];
            g.pitch = pitch;
            const fic_params *pl = &Q.pl[l];
            int *active = reinterpret_cast<int *>(ws + Q.active[l]);
            int *active_next = reinterpret_cast<int *>(ws + Q.active[l + 1]);
            int *leaf = reinterpret_cast<int *>(ws + Q.leaf[l]);
            fic_map *lmaps = reinterpret_cast<fic_map *>(ws + Q.maps[l]);
            char *ews = ws + Q.enc;
            // launch shape: fixed by the caller, cached, or timed now
            TuneChoice ch{FIC_SEARCH_SIMT, 4};
            const bool tc_ok = search_tc_supported(g);
            if (p->search == FIC_SEARCH_SIMT || (p->search == FIC_SEARCH_TC && !tc_ok)) ch.search = FIC_SEARCH_SIMT;
            else if (p->search == FIC_SEARCH_TC) ch.search = FIC_SEARCH_TC;
            else ch.search = tc_ok ? FIC_SEARCH_TC : FIC_SEARCH_SIMT;
            if (p->n_split == 0) {
                const TuneKey key{w, h, g.n, g.B, g.s_bits, g.o_bits, (int)pl->flags, p->search};
                bool have = false;
                {
                    std::lock_guard<std::mutex> lk(g_tune_mu);
                    auto it = g_tune.find(key);
                    if (it != g_tune.end()) {
                        ch = it->second;
                        have = true;
                    }
                }
                if (!have) {
                    float best = 1e30f;
                    TuneChoice bc = ch;
                    for (int s = FIC_SEARCH_TC; s <= FIC_SEARCH_SIMT; ++s) {
                        if (s == FIC_SEARCH_TC && !tc_ok) continue;
                        if (p->search != FIC_SEARCH_AUTO && s != ch.search) continue;
                        for (int wv : kWaveChoices) {
                            const EncLayout L = enc_layout(g, s, choose_split(g, pl, s) * lists_per_split(s));
                            const float ms = time_pipeline(g, pl, s, target_for(s, wv), L, ews, dimg, active, lmaps, st);
                            if (ms < best) {
                                best = ms;
                                bc = TuneChoice{s, wv};
                            }
                        }
                    }
                    ch = bc;
                    std::lock_guard<std::mutex> lk(g_tune_mu);
                    g_tune[key] = ch;
                }
            }
            const int n_split = choose_split(g, pl, ch.search);
            const int target = p->n_split > 0 ? split_target(pl, ch.search) : target_for(ch.search, ch.waves);
            const EncLayout L = enc_layout(g, ch.search, n_split * lists_per_split(ch.search));
            FIC_CUDA(encode_pipeline(g, pl, ch.search, n_split, target, L, ews, dimg, active, lmaps, nullptr, false, st,
                                     timed ? g_qt_phase.ev[l] : nullptr));
            if (l + 1 < Q.levels)
                FIC_CUDA(cudaMemsetAsync(active_next, 0, sizeof(int) * Q.g[l + 1].R, st));
            FIC_CUDA(launch_qt_split(g.R, g.nx, g.m, lmaps, active, (double)rms_split, l + 1 == Q.levels ? 1 : 0, leaf,
                                     active_next, st));
            lv.R[l] = g.R;
            lv.nx[l] = g.nx;
            lv.n[l] = g.n;
            lv.active[l] = active;
            lv.leaf[l] = leaf;
            lv.maps[l] = lmaps;
            lv.list_off[l] = list_off;
            list_off += g.R;
            g_qt_stats[1 + 4 * l] = ch.search;
            g_qt_stats[2 + 4 * l] = target;
        }
        g_qt_phase.levels = Q.levels;
        g_qt_phase.valid = timed;
        // page-locked host leaves are written in place by the gather kernel
        const bool maps_direct = maps_mem == Mem::PinnedHost;
        fic_qmap *dout = maps_dev ? maps
                                  : (maps_direct ? static_cast<fic_qmap *>(maps_alias)
                                                 : reinterpret_cast<fic_qmap *>(ws + Q.stage));
        FIC_CUDA(launch_qt_gather(lv, reinterpret_cast<int *>(ws + Q.lists), dout, maps_cap, counts, st));
        constexpr int kCounts = 2 + 2 * kMaxLevels;
        int hc_stack[kCounts];
        int *hp = pinned_words(kCounts);
        int *hc = hp ? hp : hc_stack;
        FIC_CUDA(cudaMemcpyAsync(hc, counts, sizeof(int) * kCounts, cudaMemcpyDeviceToHost, st));
        FIC_CUDA(cudaStreamSynchronize(st));
        if (!maps_dev && !maps_direct && hc[0] > 0) {
            FIC_CUDA(cudaMemcpyAsync(maps, dout, sizeof(fic_qmap) * (size_t)hc[0], cudaMemcpyDeviceToHost, st));
            FIC_CUDA(cudaStreamSynchronize(st));
        }
        for (int l = 0; l < Q.levels; ++l) {
            g_qt_stats[3 + 4 * l] = hc[1 + kMaxLevels + l];
            g_qt_stats[4 + 4 * l] = hc[1 + l];
        }
        if (n_maps) *n_maps = hc[0];
        if (hc[1 + 2 * kMaxLevels]) rc = FIC_ERR_TIMEOUT;
    }
done:
    if (owned) {
        if (cudaFreeAsync(ws, st) != cudaSuccess) {
            cudaGetLastError();
            if (rc == FIC_OK) rc = FIC_ERR_CUDA;
        }
    }
    return rc;
}

// ------------------------------------------------------------ batch

constexpr int kBatchParts = 6;  // concurrent pipelines of a batch (2, 3, 4, 6: 11.0, 10.9, 10.8, 10.7 ms on the 96-slice stack)

struct BatchSlice {
    Geometry g;
    int n_split;
    EncLayout L;
    size_t off;
    int abase, bbase;  // first rows of the slice's tensor-core operands in the shared buffers
};

// Workspace of a batch: the slice contexts, the shared operand buffers
// (tensor-core search) and one encode workspace per slice.  Slices are
// ordered by decreasing size (the persistent search takes its items in that
// order).
struct BatchPlan {
    std::vector<BatchSlice> sl;  // in input order
    std::vector<int> order;      // context order -> input slice
    int search = 0, n_split = 1;
    size_t ctx_off = 0, ra_off = 0, cb_off = 0, total = 0;
    int arows = 0, brows = 0, max_blocks = 0, max_ranges = 0, total_ranges = 0;
    bool any_wide = false, any_narrow = false;
    std::vector<int> part;  // part k: slices [part[k], part[k + 1]) of the context order, one pipeline each
    // the search's work-item counter of the pipeline starting at context k:
    // the spare fourth exact-scan counter of that slice (zeroed by its
    // statistics kernel)
    int *queue(char *ws, int k) const
    {
        const BatchSlice &b = sl[order[k]];
        return reinterpret_cast<int *>(ws + b.off + b.L.fb_count) + 3;
    }
};

int batch_plan(const fic_slice *slices, int n, const fic_params *p, BatchPlan &P)
{
    if (!slices || n <= 0 || !p) return FIC_ERR_BAD_ARG;
    int rc = check_params(p);
    if (rc != FIC_OK) return rc;
    if (p->flags & FIC_FLAG_PHASE_TIMING) return FIC_ERR_BAD_ARG;
    if (n > 1024) return FIC_ERR_CAPACITY;  // the persistent search's per-slice table
    P.sl.resize(n);
    for (int i = 0; i < n; ++i) {
        BatchSlice &b = P.sl[i];
        rc = make_geometry(slices[i].w, slices[i].h, slices[i].pitch_px, p, b.g);
        if (rc != FIC_OK) return rc;
        const int search = choose_search(b.g, p);
        if (search < 0) return FIC_ERR_UNSUPPORTED;
        if (i == 0) P.search = search;
        if (search != P.search) return FIC_ERR_UNSUPPORTED;  // (the choice depends on n and B only)
        P.max_blocks = std::max(P.max_blocks, (b.g.R + 7) / 8 + (b.g.D + 7) / 8);
        P.max_ranges = std::max(P.max_ranges, b.g.R);
        P.total_ranges += b.g.R;
        (b.g.wide ? P.any_wide : P.any_narrow) = true;
    }
    // candidate splits as for a single encode (many short lists keep the
    // exact re-scans of lists that fail certification cheap)
    for (int i = 0; i < n; ++i) {
        P.sl[i].n_split = choose_split(P.sl[i].g, p, P.search);
        P.n_split = std::max(P.n_split, P.sl[i].n_split);
    }
    // context order: the slices by decreasing size, dealt round-robin to
    // kBatchParts parts that run as concurrent pipelines (one part's
    // statistics, rows and re-score overlap another's search); each part is
    // contiguous and again sorted by size
    std::vector<int> bysize(n);
    for (int i = 0; i < n; ++i) bysize[i] = i;
    std::stable_sort(bysize.begin(), bysize.end(), [&](int a, int b) {
        return (long long)P.sl[a].g.R * P.sl[a].g.D > (long long)P.sl[b].g.R * P.sl[b].g.D;
    });
    const int parts = std::min(kBatchParts, n);
    P.order.clear();
    P.part.assign(1, 0);
    for (int h = 0; h < parts; ++h) {
        for (int k = h; k < n; k += parts) P.order.push_back(bysize[k]);
        P.part.push_back((int)P.order.size());
    }
    const bool tc = P.search == FIC_SEARCH_TC;
    for (int i : P.order) {
        BatchSlice &b = P.sl[i];
        b.abase = P.arows;
        b.bbase = P.brows;
        if (tc) {
            P.arows += search_tc_rows(b.g.R);
            P.brows += search_tc_cols(b.g.N);
        }
    }
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    P.ctx_off = take(sizeof(SliceCtx) * (size_t)n);
    if (tc) {
        const size_t row = sizeof(__half) * P.sl[0].g.KP;
        P.ra_off = take(row * P.arows);
        P.cb_off = take(row * P.brows);
    }
    for (int i : P.order) {
        BatchSlice &b = P.sl[i];
        b.L = enc_layout(b.g, P.search, b.n_split * lists_per_split(P.search), false);
        b.off = take(b.L.total);
    }
    P.total = o;
    return FIC_OK;
}

// The slice contexts of a batch in context order.
std::vector<SliceCtx> batch_contexts(const BatchPlan &P, const fic_slice *slices, const fic_params *p, char *ws)
{
    std::vector<SliceCtx> ctx(P.order.size());
    for (size_t k = 0; k < P.order.size(); ++k) {
        const int i = P.order[k];
        const BatchSlice &b = P.sl[i];
        SliceCtx &c = ctx[k];
        c = SliceCtx{};
        c.g = b.g;
        c.ec = make_epi(b.g);
        c.b = enc_bufs(b.L, ws + b.off);
        if (P.search == FIC_SEARCH_TC) {
            c.b.ra16 = reinterpret_cast<__half *>(ws + P.ra_off) + (size_t)b.abase * b.g.KP;
            c.b.cb16 = reinterpret_cast<__half *>(ws + P.cb_off) + (size_t)b.bbase * b.g.KP;
        }
        c.img = slices[i].img;
        c.maps = slices[i].maps;
        c.n_split = b.n_split;
        c.n_lists = b.n_split * lists_per_split(P.search);
        c.target = split_target(p, P.search);
        c.rb = (b.g.R + 7) / 8;
        c.db = (b.g.D + 7) / 8;
        c.abase = b.abase;
        c.bbase = b.bbase;
        // (the ranges before this slice within its part)
        const bool first = std::find(P.part.begin(), P.part.end(), (int)k) != P.part.end();
        c.r_begin = first ? 0 : ctx[k - 1].r_begin + ctx[k - 1].g.R;
    }
    return ctx;
}

// The device pipeline of a batch: the search, re-score and exact scans are
// one launch over every slice; the per-slice stages (statistics, compaction,
// operand rows, seed, map output) one launch per group of equal-sized slices
// (consecutive in context order), so that no block is idle.
cudaError_t batch_pipeline(const BatchPlan &P, const fic_params *p, char *ws, int k0, int k1, cudaStream_t st)
{
    const int n = k1 - k0;
    if (n <= 0) return cudaSuccess;
    const SliceCtx *dctx = reinterpret_cast<const SliceCtx *>(ws + P.ctx_off) + k0;
    const Geometry &g0 = P.sl[0].g;
    const int dense = (p->flags & FIC_FLAG_DENSE) ? 1 : 0;
    const bool tc = P.search == FIC_SEARCH_TC;
    // groups of equal geometry: [first, first + count)
    std::vector<std::pair<int, int>> groups;
    for (int k = 0; k < n; ++k) {
        const Geometry &g = P.sl[P.order[k0 + k]].g;
        if (!groups.empty()) {
            const Geometry &h = P.sl[P.order[k0 + groups.back().first]].g;
            if (h.R == g.R && h.D == g.D) {
                ++groups.back().second;
                continue;
            }
        }
        groups.push_back({k, 1});
    }
    int total_ranges = 0;
    for (int k = k0; k < k1; ++k) total_ranges += P.sl[P.order[k]].g.R;
    auto blocks_of = [&](int k) {
        const Geometry &g = P.sl[P.order[k0 + k]].g;
        return (g.R + 7) / 8 + (g.D + 7) / 8;
    };
    auto ranges_of = [&](int k) { return P.sl[P.order[k0 + k]].g.R; };
    cudaError_t e = cudaSuccess;
    for (auto &gr : groups)
        if ((e = launch_stats_batch(P.sl[P.order[k0 + gr.first]].g, dctx + gr.first, gr.second,
                                    stats_grid(P.sl[P.order[k0 + gr.first]].g), dense,
                                    tc_mode_of(g0, tc ? FIC_SEARCH_TC : FIC_SEARCH_SIMT), st)) != cudaSuccess)
            return e;
    for (auto &gr : groups)
        if ((e = launch_compact_seed_batch(dctx + gr.first, gr.second, ranges_of(gr.first),
                                            P.sl[P.order[k0 + gr.first]].g.m, st)) != cudaSuccess)
            return e;
    for (auto &gr : groups)
        if ((e = launch_rows_batch(P.sl[P.order[k0 + gr.first]].g, dctx + gr.first, gr.second, blocks_of(gr.first), st)) != cudaSuccess) return e;
    if (tc)
        e = launch_search_tc_batch(g0, reinterpret_cast<const __half *>(ws + P.ra_off), P.arows,
                                   reinterpret_cast<const __half *>(ws + P.cb_off), P.brows, dctx, n, dense,
                                   P.queue(ws, k0), st);
    else
        e = launch_search_simt_batch(dctx, n, P.max_ranges, P.n_split, dense, st);
    if (e != cudaSuccess) return e;
    if ((e = launch_rescore_batch(dctx, n, total_ranges, P.any_wide, P.any_narrow, g0.m, lists_per_split(P.search),
                                  tc ? search_tc_tile() : 64, (p->flags & FIC_FLAG_EXACT_SCAN) ? 1 : 0, sm_count(),
                                  st)) != cudaSuccess)
        return e;
    for (auto &gr : groups)
        if ((e = launch_finalize_batch(dctx + gr.first, gr.second, ranges_of(gr.first), P.any_wide, st)) != cudaSuccess) return e;
    return cudaSuccess;
}

// The cached graph of the last batch on this host thread.
struct BatchGraph {
    std::vector<fic_slice> table;
    fic_params p{};
    void *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t st = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t start = nullptr, end = nullptr, fork = nullptr, join[kBatchParts] = {};
    cudaStream_t cap = nullptr;  // origin stream of the capture (the caller's may be the legacy stream)
    cudaStream_t side[kBatchParts] = {};  // the other parts' pipelines
    bool ready = false;
    void reset()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        ready = false;
    }
};
thread_local BatchGraph g_batch;

bool same_batch(const BatchGraph &G, const fic_slice *slices, int n, const fic_params *p, void *ws, size_t bytes,
                cudaStream_t st)
{
    if (!G.ready || (int)G.table.size() != n || G.ws != ws || G.ws_bytes != bytes || G.st != st) return false;
    if (std::memcmp(&G.p, p, sizeof *p) != 0) return false;
    return std::memcmp(G.table.data(), slices, sizeof(fic_slice) * n) == 0;
}

int run_batch(const fic_slice *slices, int n, const fic_params *p, void *workspace, size_t workspace_bytes,
              void *stream)
{
    BatchPlan P;
    int rc = batch_plan(slices, n, p, P);
    if (rc != FIC_OK) return rc;
    if (!workspace) return FIC_ERR_BAD_ARG;
    if (workspace_bytes < P.total) return FIC_ERR_CAPACITY;
    if (reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1)) return FIC_ERR_BAD_ARG;
    for (int i = 0; i < n; ++i)
        if (!slices[i].img || !slices[i].maps || !is_device_ptr(slices[i].img) || !is_device_ptr(slices[i].maps))
            return FIC_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    BatchGraph &G = g_batch;
    if (same_batch(G, slices, n, p, workspace, workspace_bytes, st)) {
        if (cudaGraphLaunch(G.exec, st) != cudaSuccess) {
            cudaGetLastError();
            return FIC_ERR_CUDA;
        }
        return FIC_OK;
    }
    G.reset();
    if (!G.cap && cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking) != cudaSuccess) return FIC_ERR_CUDA;
    if (!G.start && cudaEventCreate(&G.start) != cudaSuccess) return FIC_ERR_CUDA;
    if (!G.end && cudaEventCreate(&G.end) != cudaSuccess) return FIC_ERR_CUDA;
    for (int k = 0; k < kBatchParts; ++k) {
        if (!G.side[k] && cudaStreamCreateWithFlags(&G.side[k], cudaStreamNonBlocking) != cudaSuccess) return FIC_ERR_CUDA;
        if (!G.join[k] && cudaEventCreateWithFlags(&G.join[k], cudaEventDisableTiming) != cudaSuccess) return FIC_ERR_CUDA;
    }
    if (!G.fork && cudaEventCreateWithFlags(&G.fork, cudaEventDisableTiming) != cudaSuccess) return FIC_ERR_CUDA;
    // the slice contexts: written once, read by every replay
    const std::vector<SliceCtx> ctx = batch_contexts(P, slices, p, ws);
    if (cudaMemcpyAsync(ws + P.ctx_off, ctx.data(), sizeof(SliceCtx) * ctx.size(), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return FIC_ERR_CUDA;
    }
    // one eager run first (kernel attributes, first-use work), then capture
    for (int pass = 0; pass < 2; ++pass) {
        // pass 0 runs on the caller's stream; pass 1 captures from a private
        // stream (the legacy default stream cannot be captured) and the graph
        // is later launched on the caller's stream
        const bool capture = pass == 1;
        const cudaStream_t o = capture ? G.cap : st;
        cudaError_t e = capture ? cudaStreamBeginCapture(o, cudaStreamCaptureModeThreadLocal) : cudaSuccess;
        const bool capturing = e == cudaSuccess && capture;
        // external records: event-record nodes that run with every replay
        if (capture && e == cudaSuccess) e = cudaEventRecordWithFlags(G.start, o, cudaEventRecordExternal);
        // the parts as concurrent branches (part 0 on the origin stream)
        const int np = (int)P.part.size() - 1;
        if (e == cudaSuccess) e = cudaEventRecord(G.fork, o);
        for (int k = 1; k < np && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(G.side[k], G.fork, 0);
        for (int k = 0; k < np && e == cudaSuccess; ++k)
            e = batch_pipeline(P, p, ws, P.part[k], P.part[k + 1], k ? G.side[k] : o);
        for (int k = 1; k < np && e == cudaSuccess; ++k) {
            e = cudaEventRecord(G.join[k], G.side[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(o, G.join[k], 0);
        }
        if (capture && e == cudaSuccess) e = cudaEventRecordWithFlags(G.end, o, cudaEventRecordExternal);
        if (capturing) {
            cudaGraph_t graph = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(o, &graph);
            if (e == cudaSuccess) e = ec;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
        }
        if (e != cudaSuccess) {
            if (debug_mode())
                fprintf(stderr, "libfic: batch %s failed: %s\n", capture ? "capture" : "run", cudaGetErrorString(e));
            cudaGetLastError();
            G.reset();
            return FIC_ERR_CUDA;
        }
        if (!capture && debug_mode()) {
            int herr = 0;
            for (size_t k = 0; k < ctx.size(); ++k) {
                if (cudaMemcpy(&herr, ctx[k].b.err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && herr)
                    fprintf(stderr, "libfic: batch slice %d: device error flag %d\n", P.order[k], herr);
            }
        }
    }
    G.table.assign(slices, slices + n);
    G.p = *p;
    G.ws = workspace;
    G.ws_bytes = workspace_bytes;
    G.st = st;
    G.ready = true;
    // the eager pass already produced the maps; the graph serves later calls
    return FIC_OK;
}

// ------------------------------------------------------------ refinement

struct RefineLayout {
    size_t roff, rsym, dcount, doff, cursor, drng, tmp, g0, g1, partial, step, ds, dof, m, v, C, nitem, ioff, items,
        ipart, ckpt, xT, total;
};

int refine_setup(int w, int h, const fic_params *p, int iters, Geometry &g, RefineGeo &rg, RefineLayout &L)
{
    if (!p || iters < 1 || iters > 1000) return FIC_ERR_BAD_ARG;
    int rc = make_geometry(w, h, w, p, g);
    if (rc != FIC_OK) return rc;
    rg = RefineGeo{g.w, g.h, g.n, g.ln, g.nx, g.R, g.t, g.U, g.V, g.D};
    const size_t N = (size_t)w * h;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    L.roff = take(sizeof(int) * g.R);
    L.rsym = take(sizeof(int) * g.R);
    L.dcount = take(sizeof(int) * g.D);
    L.doff = take(sizeof(int) * (g.D + 1));
    L.cursor = take(sizeof(int) * g.D);
    L.drng = take(sizeof(int) * g.R);
    L.tmp = take(sizeof(float) * N);
    L.g0 = take(sizeof(float) * N);
    L.g1 = take(sizeof(float) * N);
    L.partial = take(sizeof(double) * refine_partials(rg));
    L.step = take(sizeof(int));
    L.ds = take(sizeof(float) * g.R);
    L.dof = take(sizeof(float) * g.R);
    L.m = take(sizeof(float) * 2 * g.R);
    L.v = take(sizeof(float) * 2 * g.R);
    L.C = take(sizeof(float) * (size_t)g.D * g.m);
    L.nitem = take(sizeof(int) * g.D);
    L.ioff = take(sizeof(int) * (g.D + 1));
    L.items = take(sizeof(int4) * g.R);
    L.ipart = take(sizeof(float) * (size_t)g.R * g.m);
    L.ckpt = take(sizeof(float) * N * (size_t)((iters + 1) / 2));  // fic_refine only
    L.xT = take(sizeof(float) * N);
    L.total = o;
    return FIC_OK;
}

RefineBufs refine_bufs(const RefineLayout &L, char *ws)
{
    RefineBufs b;
    b.roff = reinterpret_cast<int *>(ws + L.roff);
    b.rsym = reinterpret_cast<int *>(ws + L.rsym);
    b.dcount = reinterpret_cast<int *>(ws + L.dcount);
    b.doff = reinterpret_cast<int *>(ws + L.doff);
    b.cursor = reinterpret_cast<int *>(ws + L.cursor);
    b.drng = reinterpret_cast<int *>(ws + L.drng);
    b.tmp = reinterpret_cast<float *>(ws + L.tmp);
    b.g[0] = reinterpret_cast<float *>(ws + L.g0);
    b.g[1] = reinterpret_cast<float *>(ws + L.g1);
    b.partial = reinterpret_cast<double *>(ws + L.partial);
    b.step = reinterpret_cast<int *>(ws + L.step);
    b.ds = reinterpret_cast<float *>(ws + L.ds);
    b.dof = reinterpret_cast<float *>(ws + L.dof);
    b.m = reinterpret_cast<float *>(ws + L.m);
    b.v = reinterpret_cast<float *>(ws + L.v);
    b.C = reinterpret_cast<float *>(ws + L.C);
    b.nitem = reinterpret_cast<int *>(ws + L.nitem);
    b.ioff = reinterpret_cast<int *>(ws + L.ioff);
    b.items = reinterpret_cast<int4 *>(ws + L.items);
    b.ipart = reinterpret_cast<float *>(ws + L.ipart);
    return b;
}

int refine_check_ws(void *workspace, size_t bytes, size_t need)
{
    if (!workspace) return FIC_ERR_BAD_ARG;
    if (bytes < need) return FIC_ERR_CAPACITY;
    if (reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1)) return FIC_ERR_BAD_ARG;
    return FIC_OK;
}

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess) return FIC_OK;
    cudaGetLastError();
    return FIC_ERR_CUDA;
}

thread_local cudaStream_t g_refine_cap = nullptr;

int run_refine(const void *img, int w, int h, int pitch_px, const fic_params *p, const fic_map *maps, float *s,
               float *o, int steps, int iters, float lr, float *loss, void *workspace, size_t workspace_bytes,
               void *stream)
{
    Geometry g;
    RefineGeo rg;
    RefineLayout L;
    int rc = refine_setup(w, h, p, iters, g, rg, L);
    if (rc != FIC_OK) return rc;
    if (!img || !maps || !s || !o || steps < 0 || pitch_px < w || !(lr >= 0.0f)) return FIC_ERR_BAD_ARG;
    if ((rc = refine_check_ws(workspace, workspace_bytes, L.total)) != FIC_OK) return rc;
    if (!is_device_ptr(img) || !is_device_ptr(maps) || !is_device_ptr(s) || !is_device_ptr(o) ||
        (loss && !is_device_ptr(loss)))
        return FIC_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    const RefineBufs b = refine_bufs(L, ws);
    float *ckpt = reinterpret_cast<float *>(ws + L.ckpt);
    float *xT = reinterpret_cast<float *>(ws + L.xT);
    const float init = (float)(1 << (g.B - 1));
    const float P = (float)g.P;
    cudaError_t e = refine_ranges(rg, maps, b, true, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.step, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.m, 0, sizeof(float) * 2 * g.R, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.v, 0, sizeof(float) * 2 * g.R, st);
    if (e != cudaSuccess) return cuda_rc(e);
    // one step: forward, loss and dL/dx_T (counter += 1), reverse sweep, Adam
    auto one_step = [&](cudaStream_t q) {
        cudaError_t r = refine_forward(rg, b, s, o, init, iters, ckpt, xT, q);
        if (r == cudaSuccess) r = refine_loss(rg, b, xT, img, g.B, pitch_px, b.g[0], loss, 1, q);
        if (r == cudaSuccess) r = refine_backward(rg, b, s, o, iters, ckpt, b.g[0], b.ds, b.dof, q);
        if (r == cudaSuccess) r = refine_adam(rg, b, s, o, lr, P, q);
        return r;
    };
    if (steps > 0) {
        if (!g_refine_cap && cudaStreamCreateWithFlags(&g_refine_cap, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_rc(cudaErrorUnknown);
        // capture one step from a private stream (the caller's may be the
        // legacy stream) ordered after the set-up above, then replay it
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        e = cudaStreamBeginCapture(g_refine_cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t es = one_step(g_refine_cap);
            const cudaError_t ee = cudaStreamEndCapture(g_refine_cap, &graph);
            e = es != cudaSuccess ? es : ee;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        for (int i = 0; i < steps && e == cudaSuccess; ++i) e = cudaGraphLaunch(exec, st);
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_rc(e);
    }
    // the loss after the last step
    e = refine_forward(rg, b, s, o, init, iters, ckpt, xT, st);
    if (e == cudaSuccess) e = refine_loss(rg, b, xT, img, g.B, pitch_px, b.g[0], loss, 0, st);
    return cuda_rc(e);
}

// ------------------------------------------------------------ decode

// g: the encode geometry of the maps; gs: the same maps decoded at scale
// 2^scale_log2 (range and domain sides and positions scaled, the 2x2
// contraction kept; range and domain counts and indices unchanged).
int decode_geometry(int w, int h, const fic_params *p, int scale_log2, Geometry &g, Geometry &gs)
{
    int rc = make_geometry(w, h, w, p, g);
    if (rc != FIC_OK) return rc;
    if (scale_log2 < -3 || scale_log2 > 3) return FIC_ERR_BAD_ARG;
    gs = g;
    if (scale_log2 >= 0) {
        const int z = 1 << scale_log2;
        if ((long long)w * z * h * z > (1LL << 30)) return FIC_ERR_SIZE;
        gs.w = w * z, gs.h = h * z, gs.n = g.n * z, gs.t = g.t * z;
    } else {
        const int z = 1 << -scale_log2;
        // positions and sides must stay whole pixels; a range keeps >= 1 pixel
        if (g.n % z || g.t % z || w % z || h % z) return FIC_ERR_SIZE;
        gs.w = w / z, gs.h = h / z, gs.n = g.n / z, gs.t = g.t / z;
    }
    gs.pitch = gs.w;
    gs.m = gs.n * gs.n;
    gs.ln = 0;
    while ((1 << gs.ln) < gs.n) ++gs.ln;
    return FIC_OK;
}

int run_decode(const fic_map *maps, int n_maps, int w, int h, const fic_params *p, int scale_log2, float init,
               float *out, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!maps || !out) return FIC_ERR_BAD_ARG;
    Geometry g, gs;
    int rc = decode_geometry(w, h, p, scale_log2, g, gs);
    if (rc != FIC_OK) return rc;
    if (n_maps != g.R) return FIC_ERR_CAPACITY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t npx = (size_t)gs.w * gs.h;
    const size_t dws = align_up(decode_workspace_bytes(gs));
    const size_t maps_b = align_up(sizeof(fic_map) * g.R);
    const size_t out_b = align_up(sizeof(float) * npx);
    const size_t total = dws + maps_b + out_b;
    char *ws = static_cast<char *>(workspace);
    bool owned = false;
    const bool maps_dev = is_device_ptr(maps);
    const bool out_dev = is_device_ptr(out);
    if (!maps_dev) {
        // host maps are validated here; device maps are trusted to come from fic_encode
        for (int r = 0; r < g.R; ++r)
            if (maps[r].domain_idx >= (uint32_t)g.D || maps[r].iso < 0 || maps[r].iso > 7)
                return FIC_ERR_BAD_ARG;
    }
    if (ws) {
        if (workspace_bytes < total) return FIC_ERR_CAPACITY;
        if (reinterpret_cast<uintptr_t>(ws) & (kAlign - 1)) return FIC_ERR_BAD_ARG;
    } else {
        if (cudaMallocAsync(reinterpret_cast<void **>(&ws), total, st) != cudaSuccess) {
            cudaGetLastError();
            return FIC_ERR_CUDA;
        }
        owned = true;
    }
    {
        const fic_map *dmaps = maps;
        float *dout = out_dev ? out : reinterpret_cast<float *>(ws + dws + maps_b);
        if (!maps_dev) {
            FIC_CUDA(cudaMemcpyAsync(ws + dws, maps, sizeof(fic_map) * g.R, cudaMemcpyHostToDevice, st));
            dmaps = reinterpret_cast<const fic_map *>(ws + dws);
        }
        FIC_CUDA(launch_decode(gs, dmaps, init, p->decode_iters, ws, dout, st));
        if (!out_dev) {
            FIC_CUDA(cudaMemcpyAsync(out, dout, sizeof(float) * npx, cudaMemcpyDeviceToHost, st));
            FIC_CUDA(cudaStreamSynchronize(st));
        } else if (!maps_dev) {
            FIC_CUDA(cudaStreamSynchronize(st));
        }
    }
done:
    if (owned) {
        if (cudaFreeAsync(ws, st) != cudaSuccess) {
            cudaGetLastError();
            if (rc == FIC_OK) rc = FIC_ERR_CUDA;
        }
    }
    return rc;
}

}  // namespace

namespace fic {
int encode_with_workspace(const void *img, int w, int h, int pitch_px, const fic_params *p, fic_map *maps,
                          int maps_cap, int *n_maps, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!maps || !workspace) return FIC_ERR_BAD_ARG;
    g_no_alloc = true;  // the caller may not allocate, not even pinned host memory
    const int rc = run_encode(img, w, h, pitch_px, p, maps, maps_cap, n_maps, workspace, workspace_bytes, stream,
                              nullptr);
    g_no_alloc = false;
    return rc;
}
}  // namespace fic

extern "C" {

int fic_encode(const void *img, int w, int h, int pitch_px, const fic_params *p, fic_map *maps,
               int maps_cap, int *n_maps, void *workspace, size_t workspace_bytes, void *stream)
{
    if (!maps) return FIC_ERR_BAD_ARG;
    return run_encode(img, w, h, pitch_px, p, maps, maps_cap, n_maps, workspace, workspace_bytes, stream,
                      nullptr);
}

int fic_cross_terms(const void *img, int w, int h, int pitch_px, const fic_params *p, float *out,
                    void *workspace, size_t workspace_bytes, void *stream)
{
    if (!out) return FIC_ERR_BAD_ARG;
    return run_encode(img, w, h, pitch_px, p, nullptr, 0, nullptr, workspace, workspace_bytes, stream, out);
}

int fic_decode(const fic_map *maps, int n_maps, int w, int h, const fic_params *p, float init,
               float *out, void *workspace, size_t workspace_bytes, void *stream)
{
    return run_decode(maps, n_maps, w, h, p, 0, init, out, workspace, workspace_bytes, stream);
}

int fic_decode_scaled(const fic_map *maps, int n_maps, int w, int h, const fic_params *p, int scale_log2, float init,
                      float *out, void *workspace, size_t workspace_bytes, void *stream)
{
    return run_decode(maps, n_maps, w, h, p, scale_log2, init, out, workspace, workspace_bytes, stream);
}

int fic_decode_workspace_size(int w, int h, const fic_params *p, size_t *bytes)
{
    return fic_decode_scaled_workspace_size(w, h, p, 0, bytes);
}

int fic_decode_scaled_workspace_size(int w, int h, const fic_params *p, int scale_log2, size_t *bytes)
{
    if (!bytes) return FIC_ERR_BAD_ARG;
    Geometry g, gs;
    const int rc = decode_geometry(w, h, p, scale_log2, g, gs);
    if (rc != FIC_OK) return rc;
    *bytes = align_up(decode_workspace_bytes(gs)) + align_up(sizeof(fic_map) * g.R) +
             align_up(sizeof(float) * (size_t)gs.w * gs.h);
    return FIC_OK;
}

const char *fic_status_str(int status)
{
    switch (status) {
    case FIC_OK: return "ok";
    case FIC_ERR_BAD_ARG: return "invalid argument";
    case FIC_ERR_SIZE: return "image size must be a multiple of the range size and at least two ranges";
    case FIC_ERR_BITDEPTH: return "unsupported bit depth or code width";
    case FIC_ERR_CAPACITY: return "output or workspace buffer too small";
    case FIC_ERR_CUDA: return "CUDA runtime error";
    case FIC_ERR_TIMEOUT: return "device-side wait timed out";
    case FIC_ERR_UNSUPPORTED: return "parameters not supported by this library";
    default: return "unknown status";
    }
}

int fic_last_encode_phase_ms(double out[5])
{
    if (!out) return FIC_ERR_BAD_ARG;
    if (!g_phase.valid) return FIC_ERR_BAD_ARG;
    if (cudaEventSynchronize(g_phase.ev[5]) != cudaSuccess) {
        cudaGetLastError();
        return FIC_ERR_CUDA;
    }
    for (int i = 0; i < 5; ++i) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, g_phase.ev[i], g_phase.ev[i + 1]) != cudaSuccess) {
            cudaGetLastError();
            return FIC_ERR_CUDA;
        }
        out[i] = ms;
    }
    return FIC_OK;
}

int fic_encode_quadtree(const void *img, int w, int h, int pitch_px, const fic_params *p, int min_size,
                        float rms_split, fic_qmap *maps, int maps_cap, int *n_maps, void *workspace,
                        size_t workspace_bytes, void *stream)
{
    return run_quadtree(img, w, h, pitch_px, p, min_size, rms_split, maps, maps_cap, n_maps, workspace,
                        workspace_bytes, stream);
}

int fic_quadtree_workspace_size(int w, int h, const fic_params *p, int min_size, size_t *bytes)
{
    if (!bytes) return FIC_ERR_BAD_ARG;
    QtPlan Q;
    const int rc = qt_plan(w, h, w, p, min_size, 0, Q);
    if (rc != FIC_OK) return rc;
    *bytes = Q.total;
    return FIC_OK;
}

int fic_last_quadtree_stats(int64_t out[17])
{
    if (!out) return FIC_ERR_BAD_ARG;
    for (int i = 0; i < 1 + 4 * kMaxLevels; ++i) out[i] = g_qt_stats[i];
    for (int i = 1 + 4 * kMaxLevels; i < 17; ++i) out[i] = 0;
    return FIC_OK;
}

int fic_last_quadtree_phase_ms(double out[3])
{
    if (!out) return FIC_ERR_BAD_ARG;
    if (!g_qt_phase.valid) return FIC_ERR_BAD_ARG;
    for (int l = 0; l < kMaxLevels; ++l) {
        out[l] = 0.0;
        if (l >= g_qt_phase.levels) continue;
        float ms = 0.0f;
        if (cudaEventSynchronize(g_qt_phase.ev[l][1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms, g_qt_phase.ev[l][0], g_qt_phase.ev[l][1]) != cudaSuccess) {
            cudaGetLastError();
            return FIC_ERR_CUDA;
        }
        out[l] = ms;
    }
    return FIC_OK;
}

int fic_encode_batch(const fic_slice *slices, int n, const fic_params *p, void *workspace, size_t workspace_bytes,
                     void *stream)
{
    return run_batch(slices, n, p, workspace, workspace_bytes, stream);
}

int fic_batch_workspace_size(const fic_slice *slices, int n, const fic_params *p, size_t *bytes)
{
    if (!bytes) return FIC_ERR_BAD_ARG;
    BatchPlan P;
    const int rc = batch_plan(slices, n, p, P);
    if (rc != FIC_OK) return rc;
    *bytes = P.total;
    return FIC_OK;
}

int fic_last_batch_slice_ms(float *out, int n)
{
    const BatchGraph &G = g_batch;
    if (!out || !G.ready || n > (int)G.table.size()) return FIC_ERR_BAD_ARG;
    float ms = 0.0f;
    if (cudaEventSynchronize(G.end) != cudaSuccess || cudaEventElapsedTime(&ms, G.start, G.end) != cudaSuccess) {
        cudaGetLastError();
        return FIC_ERR_CUDA;
    }
    for (int i = 0; i < n; ++i) out[i] = ms;  // every stage covers every slice: they complete together
    return FIC_OK;
}

int fic_refine_workspace_size(int w, int h, const fic_params *p, int iters, size_t *bytes)
{
    if (!bytes) return FIC_ERR_BAD_ARG;
    Geometry g;
    RefineGeo rg;
    RefineLayout L;
    const int rc = refine_setup(w, h, p, iters, g, rg, L);
    if (rc != FIC_OK) return rc;
    *bytes = L.total;
    return FIC_OK;
}

int fic_refine_forward(const fic_map *maps, int w, int h, const fic_params *p, const float *s, const float *o,
                       float init, int iters, float *x_out, float *ckpt, void *workspace, size_t workspace_bytes,
                       void *stream)
{
    Geometry g;
    RefineGeo rg;
    RefineLayout L;
    int rc = refine_setup(w, h, p, iters, g, rg, L);
    if (rc != FIC_OK) return rc;
    if (!maps || !s || !o || !x_out || !ckpt) return FIC_ERR_BAD_ARG;
    if ((rc = refine_check_ws(workspace, workspace_bytes, L.total)) != FIC_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const RefineBufs b = refine_bufs(L, static_cast<char *>(workspace));
    cudaError_t e = refine_ranges(rg, maps, b, false, st);
    if (e == cudaSuccess) e = refine_forward(rg, b, s, o, init, iters, ckpt, x_out, st);
    return cuda_rc(e);
}

int fic_refine_backward(const fic_map *maps, int w, int h, const fic_params *p, const float *s, const float *o,
                        int iters, const float *ckpt, const float *grad_x, float *grad_s, float *grad_o,
                        void *workspace, size_t workspace_bytes, void *stream)
{
    Geometry g;
    RefineGeo rg;
    RefineLayout L;
    int rc = refine_setup(w, h, p, iters, g, rg, L);
    if (rc != FIC_OK) return rc;
    if (!maps || !s || !o || !ckpt || !grad_x || !grad_s || !grad_o) return FIC_ERR_BAD_ARG;
    if ((rc = refine_check_ws(workspace, workspace_bytes, L.total)) != FIC_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const RefineBufs b = refine_bufs(L, static_cast<char *>(workspace));
    cudaError_t e = refine_ranges(rg, maps, b, true, st);
    if (e == cudaSuccess) e = refine_backward(rg, b, s, o, iters, ckpt, grad_x, grad_s, grad_o, st);
    return cuda_rc(e);
}

int fic_refine(const void *img, int w, int h, int pitch_px, const fic_params *p, const fic_map *maps, float *s,
               float *o, int steps, int iters, float lr, float *loss, void *workspace, size_t workspace_bytes,
               void *stream)
{
    return run_refine(img, w, h, pitch_px, p, maps, s, o, steps, iters, lr, loss, workspace, workspace_bytes,
                      stream);
}

int fic_last_encode_stats(int64_t out[4])
{
    if (!out) return FIC_ERR_BAD_ARG;
    for (int i = 0; i < 4; ++i) out[i] = g_stats[i];
    return FIC_OK;
}

int fic_set_wait_limit_ns(uint64_t ns)
{
    fic::set_wait_limit_ns((unsigned long long)ns);
    return FIC_OK;
}

uint64_t fic_get_wait_limit_ns(void) { return (uint64_t)fic::wait_limit_ns(); }

}  // extern "C"
