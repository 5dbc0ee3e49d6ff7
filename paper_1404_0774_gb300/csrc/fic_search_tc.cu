// Tensor-core range-domain search for sm_103a (tcgen05 + TMA + TMEM).
//
// The cross term of eq 9, X = sum_i q_i b_i over all ranges x all candidates
// (domain d, symmetry k), is a dense contraction M = ranges, N = candidates,
// K = pixels.  Operands are centred integers in FP16 (exact):
//   A row (range r):      [ b'_1..b'_m | b'_1..b'_m (12-bit only) | e_hi e_lo 0.. ]
//   B row (candidate):    [ 128*hi_i   | lo_i       (12-bit only) | -16 f_d  -f_d/m 0.. ]
// with q'_i = 128*hi_i + lo_i (8-bit: a single q' block), so that the FP32
// accumulator is Xt = sum q'b' - e_r f_d / m = (m X - Sq Sb) / m.  The K
// dimension is laid out as one block per copy of the pixels (8x8 ranges:
// 64 elements, SWIZZLE_128B; 4x4 ranges: 16 elements, SWIZZLE_32B) plus one
// 16-element SWIZZLE_32B tail block carrying the centring terms.  For 12-bit
// images the hi and lo blocks go to separate TMEM accumulators, whose sums
// are exact (one MMA of 2 x 64 candidate rows per K step: a B stage holds the
// tile's hi rows and then its lo rows), and the tail's centring term is
// folded in by the epilogue.
// 16x16 ranges (K = 256 per copy): the range pixels are staged once as four
// 64-element boxes that every part's MMAs read, the candidate rows stream
// through a ring of one-box stages (a tile is parts x 4 stages), the tail is
// not used (the centring correction is applied in the epilogue), and the
// FP32 accumulation over K = 256 may round: the statistics kernel widens the
// screening allowances for it.
//
// Persistent CTA, one per SM.  A work item is a row tile of 128 screened
// ranges (one per TMEM lane) against one split of the candidate columns,
// streamed in 192-column super-tiles of three 64-column MMA tiles:
//   warp 0        TMA producer (one thread): the item queue, A once per item,
//                 B tiles into a 4-stage ring (16x16 ranges: B boxes into a
//                 7-stage ring)
//   warp 1        TMEM allocator + MMA issuer (one thread): tcgen05.mma
//                 kind::f16 128xNx16 per K step of every MMA tile into a ring
//                 of four TMEM accumulator slots
//   warps 2..13   epilogue, three per TMEM lane quadrant (three per scheduler
//                 with the register budget of 14 warps): part p takes MMA
//                 tile p of every super-tile, FP32 screening (eq 8-12 with
//                 quantisation), per-range candidate lists
// Every mbarrier wait is bounded by a wall-clock limit; on expiry the CTA sets
// an error flag, stops, drains its outstanding TMA loads (bounded), frees its
// TMEM and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <atomic>

#include "fic_internal.cuh"

namespace fic {
namespace {

constexpr int BM = 128;
constexpr int BN = 64;                          // candidates per MMA tile (B rows of one stage)
constexpr int STAGES = 4;
constexpr int NACC = 4;                         // accumulator slots (one per MMA tile in flight)
constexpr int EPI_COLS = 32;                    // columns of a tile per epilogue warp
// A work item's columns come in super-tiles of LISTS MMA tiles; epilogue
// part p (one warp per TMEM lane quadrant) takes MMA tile p of every
// super-tile, both of its 32-column chunks.  The three warps of a scheduler
// (one per part) so work on different tiles, which the MMA warp produces one
// after another into a ring of NACC accumulator slots, instead of all
// waiting for and working on the same tile at the same time; and each of
// them pays the per-tile wait, staging and release once per two chunks.
constexpr int LISTS = 3;                        // epilogue warps per TMEM lane quadrant
constexpr int SUPER = LISTS * BN;               // columns of a super-tile (the split unit)
static_assert(SUPER == 192, "active_splits and split_tile recognise the tensor-core search by its 192-column unit");
constexpr int CHUNKS = BN / EPI_COLS;           // chunks of an MMA tile per epilogue warp
constexpr int EPI_WARPS = 4 * LISTS;
constexpr int THREADS = 64 + 32 * EPI_WARPS;    // TMA warp, MMA warp, epilogue
constexpr int DC_WARP = EPI_COLS / 8;           // domains per warp per tile
// Limits of the bounded waits.  A pipeline wait (for a stage, an
// accumulator, an item) gives up after the run-time limit `wait_ns` (2 s by
// default, fic_set_wait_limit_ns); the drain at exit, which waits for copies
// and MMAs already issued (they finish in microseconds), always allows 2 s so
// that no copy or MMA can still be writing when the CTA frees its shared
// memory and TMEM.
constexpr unsigned long long kDrainNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// try_wait whose suspension is capped at `hint_ns`.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Longest suspension of one try_wait in a pipeline wait.  The thread wakes
// as soon as the phase completes, so the hint costs nothing in latency; it
// keeps a waiting role from re-issuing try_wait in a loop, which takes issue
// slots from the epilogue warps on the same scheduler (measured: 2 us less
// search time on the 512x512 slice than unhinted try_wait).
constexpr uint32_t kSuspendHintNs = 50000u;

// Limits below this are honoured to the timer's resolution: each try_wait
// suspends for at most the limit and the clock is read after every one
// (otherwise after every 64th).
constexpr unsigned long long kShortWaitNs = 1000000ull;

// Bounded wait for the phase of `parity` to complete.  Returns false when the
// CTA is aborting (another role timed out) or this wait timed out (after
// wait_ns of %globaltimer).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_s, int *err,
                                          unsigned long long wait_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    const bool short_wait = wait_ns < kShortWaitNs;
    for (uint32_t i = 1;; ++i) {
        if (short_wait ? mbar_try_wait_hint(bar, parity, (uint32_t)wait_ns)
                       : mbar_try_wait_hint(bar, parity, kSuspendHintNs))
            return true;
        if (short_wait || (i & 63) == 0) {
            if (*abort_s) return false;
            if (gtimer() - t0 > wait_ns) {
                *abort_s = 1;
                atomicExch(err, 1);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// SM100 shared-memory matrix descriptor, K-major, swizzled.
// layout: 2 = SWIZZLE_128B (SBO 1024), 6 = SWIZZLE_32B (SBO 256)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo, uint32_t layout)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;                         // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;     // stride byte offset: 8-row group pitch
    d |= (uint64_t)1u << 46;                         // descriptor version (sm_100 family)
    d |= (uint64_t)layout << 61;
    return d;
}

// Instruction descriptor: kind::f16, A = B = F16, D = F32, both K-major.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 lanes x 32 consecutive columns (one FP32 per column) for this warp's
// lane quadrant.  Asynchronous: the registers are valid after tmem_wait().
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// Wait for this thread's outstanding tcgen05.ld; the register operands tie
// every later use of r[] to the wait.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]),
                   "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]),
                   "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// Wait for this thread's outstanding tcgen05.ld of two 32-column chunks.
__device__ __forceinline__ void tmem_wait2(uint32_t (&a)[32], uint32_t (&b)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]),
                   "+r"(a[7]), "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]),
                   "+r"(a[14]), "+r"(a[15]), "+r"(a[16]), "+r"(a[17]), "+r"(a[18]), "+r"(a[19]), "+r"(a[20]),
                   "+r"(a[21]), "+r"(a[22]), "+r"(a[23]), "+r"(a[24]), "+r"(a[25]), "+r"(a[26]), "+r"(a[27]),
                   "+r"(a[28]), "+r"(a[29]), "+r"(a[30]), "+r"(a[31]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]),
                   "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]), "+r"(b[8]), "+r"(b[9]),
                   "+r"(b[10]), "+r"(b[11]), "+r"(b[12]), "+r"(b[13]), "+r"(b[14]), "+r"(b[15]), "+r"(b[16]),
                   "+r"(b[17]), "+r"(b[18]), "+r"(b[19]), "+r"(b[20]), "+r"(b[21]), "+r"(b[22]), "+r"(b[23]),
                   "+r"(b[24]), "+r"(b[25]), "+r"(b[26]), "+r"(b[27]), "+r"(b[28]), "+r"(b[29]), "+r"(b[30]),
                   "+r"(b[31])
                 :
                 : "memory");
}

// Rare pass of one 32-column chunk (warp-collective: every lane calls it):
// stage this thread's cross terms X[] in its column of the staging buffer,
// then each thread visits its own candidates of `mask`.  Staging is per
// thread, so no cross-lane ordering is needed.
__device__ __forceinline__ void rare_chunk(const float (&X)[32], uint32_t mask, const int (&od)[4],
                                           const float4 (&dc)[4], float er, float *xcol, int stride,
                                           const RangeEpi &re, const EpiConst &ec, ListState &L, int *tbest_r)
{
    if (mask) {
#pragma unroll
        for (int j = 0; j < 32; ++j) xcol[j * stride] = X[j];
        epi_rare(xcol, stride, od, dc, er, re, ec, L, mask);
        if (L.T < L.Tpub) {
            atomicMin(tbest_r, f2ord(L.T));
            L.Tpub = L.T;
        }
    }
    __syncwarp();
}

// The column constants of one domain as the tensor-core epilogue reads them
// (staged in shared memory once per tile): a = (kappa, kappa, -sqz, -sqz),
// b = (g, g, alpha, 0) with g = Sq/m - round(Sq/m), so that the centring
// correction of a range with factor e_r is corr = -e_r * g (epi_corr); each
// pair is one aligned 64-bit operand of the packed arithmetic.
struct DcPack {
    float4 a, b;
};

__device__ __forceinline__ DcPack dc_pack(const float4 &c4, const EpiConst &ec)
{
    const float a = c4.w * ec.invm;
    const float g = a - floorf(a + 0.5f);  // exact: Sq/m has at most 6 fraction bits
    DcPack d;
    d.a = make_float4(c4.z, c4.z, -c4.y, -c4.y);
    d.b = make_float4(g, g, c4.x, 0.0f);
    return d;
}

// epi_keys32<true> of fic_internal.cuh (the near-boundary candidates go to the
// rare pass, the mask is assembled from sign bits) on the packed constants,
// with the threshold folded into the key: the sign of
// lambda w^2 + (c y - thr') replaces that of (c y + lambda w^2) - thr, one
// instruction less per pair of candidates.  The mask only chooses what the
// rare pass visits (which recomputes each key as epi_key does), so it may hold
// more candidates, never fewer: with P = c y and Q = (lambda w) w exact, the
// key k = RN(Q + RN(P)) is below thr only if P + Q < thr + u(|P| + |thr|);
// near the sign change |P| <= |thr'| + qmax, so thr' = thr + 2^-21 (|thr| +
// qmax) exceeds every rounding of both forms (u = 2^-24) and
// RN(Q + RN(P - thr')) < 0 whenever k < thr.  kZero: add the penalty to
// s-code-0 keys (zp); the caller takes the variant without it when no lane of
// the warp can list an s-code-0 candidate (the key of every s-code-0
// candidate of a range is the same value K0; without the penalty those keys
// stay K0, and K0 >= thr keeps them out of the mask as the penalty would).
template <bool kZero>
__device__ __forceinline__ uint32_t epi_keys32_tc(const float (&X)[32], const DcPack *dp, float zb, float rho_lim,
                                                  f32x2_t er2, const EpiConst &ec, float thr, float zp)
{
    uint32_t mask = 0, far = 0;  // bit-reversed masks of k < thr, of |rho| below the band
    const float thr_up = __fadd_ru(thr, __fmul_ru(__fadd_ru(fabsf(thr), ec.qmax), 4.76837158203125e-07f));  // 2^-21
    const f32x2_t mthr = pk2(-thr_up, -thr_up);
    const float mlim2 = -__fmul_rd(rho_lim, rho_lim);
    const f32x2_t mlim = pk2(mlim2, mlim2);
    const f32x2_t two_ls = pk2(ec.two_ls, ec.two_ls), mls = pk2(-ec.ls, -ec.ls);
    const f32x2_t mag = pk2(kMagic, kMagic), zb2 = pk2(zb, zb), invg = pk2(ec.invG, ec.invG);
    const f32x2_t mg = pk2(-ec.G, -ec.G), lam = pk2(ec.lambda, ec.lambda), zpp = pk2(zp, zp);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 A = dp[q].a, Bv = dp[q].b;
        const f32x2_t kap = pk2(A.x, A.y), msqz = pk2(A.z, A.w);
        const f32x2_t mcorr = mul2(er2, pk2(Bv.x, Bv.y));  // -corr in both halves
        float mc, mc1;
        upk2(mcorr, mc, mc1);
        const float alpha = Bv.z;
        const float bq = fmaf(-mc, alpha, 0.5f);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int j = q * 8 + 2 * h;
            const float u0 = __saturatef(fmaf(X[j], alpha, bq));
            const float u1 = __saturatef(fmaf(X[j + 1], alpha, bq));
            const f32x2_t x = pk2(X[j], X[j + 1]);
            const f32x2_t r = fma2(pk2(u0, u1), two_ls, mls);  // Ls * clamp(s, -1, 1)
            const f32x2_t c = sub2(add2(r, mag), mag);          // rounded code
            const f32x2_t rho = sub2(r, c);
            const f32x2_t z = fma2(c, msqz, zb2);
            const f32x2_t e = sub2(fma2(z, invg, mag), mag);
            const f32x2_t wv = fma2(e, mg, z);
            const f32x2_t y = fma2(c, kap, sub2(mcorr, x));
            f32x2_t d = fma2(mul2(wv, lam), wv, fma2(c, y, mthr));  // key - thr'
            if (kZero) {
                float c0, c1;
                upk2(c, c0, c1);
                const float zero0 = __saturatef(fmaf(c0, -c0, 1.0f));  // 1 for c = 0, else 0
                const float zero1 = __saturatef(fmaf(c1, -c1, 1.0f));
                d = fma2(pk2(zero0, zero1), zpp, d);
            }
            float d0, d1, t0, t1;
            upk2(d, d0, d1);
            upk2(fma2(rho, rho, mlim), t0, t1);
            mask = __funnelshift_l(__float_as_uint(d0), mask, 1);  // (mask << 1) | sign bit
            mask = __funnelshift_l(__float_as_uint(d1), mask, 1);
            far = __funnelshift_l(__float_as_uint(t0), far, 1);
            far = __funnelshift_l(__float_as_uint(t1), far, 1);
        }
    }
    return __brev(mask | ~far);
}

// Bits of the first nv (1..32) columns of a 32-column chunk.
__device__ __forceinline__ uint32_t col_mask(int nv) { return nv >= 32 ? 0xffffffffu : (1u << nv) - 1u; }

struct TcMaps {
    CUtensorMap a128, a32, b128, b32;
};

}  // namespace

// NBLK: number of pixel K blocks (1 for 8-bit, 2 for 12-bit); BW: their width.
// dump != nullptr: write the raw accumulators Xt[r][c] instead of screening.
constexpr int kItemQ = 4;  // work items handed from the TMA warp to the other roles

// Work item of the persistent search: row tile `r0` of slice `s` against the
// candidate tiles [t_begin, t_end) of split `split`.
struct TcItem {
    int s, r0, split, t_begin, t_end;
};

// Work item `item` (ip_s: per-slice prefix of the items, ns_s / rt_s: active
// splits / row tiles per slice).  Items are numbered slice by slice, split
// major: the row tiles of a split run side by side, and later splits start
// from the best keys the earlier ones shared.
__device__ __forceinline__ TcItem tc_item(const SliceCtx *ctx, const int *ip_s, const int *ns_s, const int *rt_s,
                                          int n, int item)
{
    int lo = 0, hi = n - 1;  // the last slice with ip_s[s] <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ip_s[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    TcItem it;
    it.s = lo;
    const int local = item - ip_s[lo], ns = ns_s[lo], nrt = rt_s[lo];
    it.split = local / nrt;
    it.r0 = (local - it.split * nrt) * BM;
    const int ncol = 8 * ctx[lo].b.cb.counts[2];
    const int tiles = (ncol + SUPER - 1) / SUPER;
    it.t_begin = split_tile(tiles, it.split, ns, SUPER);
    it.t_end = split_tile(tiles, it.split + 1, ns, SUPER);
    return it;
}

// Persistent tensor-core search over the work items of n slices (n = 1: a
// single encode); every role (TMA producer, MMA issuer, epilogue warps) walks
// the same item sequence, so the pipelines run on across item boundaries.
template <int NBLK, int BW, int KB, bool BATCH>
__device__ __forceinline__ void search_tc_run(const TcMaps &maps, const SliceCtx &one, const SliceCtx *many, int n,
                                              int dense, float *dump, uint32_t smem_bytes, int *queue,
                                              unsigned long long wait_ns)
{
    // a single search reads its context from the kernel parameters (constant
    // bank operands in the epilogue's inner loop)
    const SliceCtx *ctx = BATCH ? many : &one;
    // BW: K elements per copy of the pixels (64: 128B-swizzled blocks, n = 8;
    // 16: 32B-swizzled blocks, n = 4); KPB MMAs of K = 16 per block
    constexpr int KPB = BW / 16;
    constexpr uint32_t A_BLK = BM * BW * 2;              // bytes of one block, A
    constexpr uint32_t B_BLK = BN * BW * 2;
    // KB == 1 (4x4 and 8x8 ranges): A holds NBLK copies of the range pixels
    // and the tail; a B stage holds a whole tile (NBLK blocks and the tail).
    // KB > 1 (16x16 ranges, K = 256 per part): A holds the range pixels once,
    // KB boxes of 64 (every part's MMAs read them); a B stage holds one box
    // of one part, a tile is NBLK * KB stages, and there is no tail (the
    // centring correction is applied in the epilogue).
    constexpr uint32_t A_BYTES = KB == 1 ? NBLK * A_BLK + BM * 32 : KB * A_BLK;
    constexpr uint32_t B_BYTES = KB == 1 ? NBLK * B_BLK + BN * 32 : B_BLK;
    constexpr int NSTG = KB == 1 ? STAGES : 7;  // stages of the B ring
    constexpr int KSTEPS = NBLK * KPB + 1;
    constexpr uint32_t SBO = BW == 64 ? 1024 : 256, LAYOUT = BW == 64 ? 2 : 6;
    constexpr uint32_t IDESC = instr_desc(BM, BN);
    constexpr uint32_t IDESC2 = instr_desc(BM, 2 * BN);  // 12-bit: a stage's hi and lo rows as one operand
    // 12-bit: the hi and lo parts of q' accumulate separately (each sum is
    // exact in FP32: multiples of 128 below 2^31, integers below 2^23) and the
    // centring correction is folded into the epilogue, so the only rounding
    // of the cross term is that of hi + lo.  8-bit: one accumulator, tail
    // columns included.
    constexpr uint32_t PARTS = NBLK == 2 ? 2 : 1;
    // the centring correction -e_r f_d / m is added in the epilogue (else by
    // the tail MMA)
    constexpr bool CORR_EPI = PARTS == 2 || KB > 1;
    constexpr uint32_t ACC_COLS = BN * PARTS;
    // bytes the MMAs read (the expected transaction counts): 12-bit items load
    // only A block 0 (both parts multiply the same range pixels) and no tail
    // boxes (the correction is the epilogue's)
    constexpr uint32_t A_TX = KB > 1 ? KB * A_BLK : (PARTS == 2 ? A_BLK : NBLK * A_BLK + BM * 32);
    constexpr uint32_t B_TX = KB > 1 ? B_BLK : (CORR_EPI ? NBLK * B_BLK : NBLK * B_BLK + BN * 32);
    constexpr uint32_t TMEM_COLS = ACC_COLS * NACC <= 256 ? 256 : 512;  // allocation: a power of two

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = smem;
    uint8_t *sB = smem + A_BYTES;  // A_BYTES is a multiple of 1024
    constexpr int ET = 32 * EPI_WARPS;                                // epilogue threads
    float *xsm = reinterpret_cast<float *>(sB + NSTG * B_BYTES);  // [32][ET] cross terms (rare pass)
    float4 *dcs = reinterpret_cast<float4 *>(xsm + 32 * ET);        // [EPI_WARPS][DC_WARP] domain constants
    // then [EPI_WARPS][DC_WARP] original domain ids, then the packed constants
    DcPack *dps = reinterpret_cast<DcPack *>(reinterpret_cast<int *>(dcs + EPI_WARPS * DC_WARP) + EPI_WARPS * DC_WARP);
    __shared__ __align__(8) uint64_t full_bar[NSTG], empty_bar[NSTG], a_full, a_empty, tfull_bar[NACC],
        tempty_bar[NACC];
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;
    constexpr int NSL = BATCH ? kMaxBatch : 1;  // slices of the launch
    __shared__ int ip_s[NSL + 1], ns_s[NSL], rt_s[NSL];
    __shared__ int item_q[kItemQ];
    __shared__ __align__(8) uint64_t q_full[kItemQ], q_empty[kItemQ];

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    // A single search runs the set-up that reads nothing an earlier kernel
    // writes -- the barriers, the TMEM allocation, the tensor-map descriptors
    // -- before the wait for that kernel, so that it overlaps its tail (slice
    // encode 2.6 us shorter).  A batch waits first: its search shares the SMs
    // with the other pipelines of the graph (measured 4.6 % slower otherwise).
    if constexpr (BATCH) grid_dep_sync();
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTG; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&a_full, 1);
        mbar_init(&a_empty, 1);
        for (int q = 0; q < kItemQ; ++q) {
            mbar_init(&q_full[q], 1);
            mbar_init(&q_empty[q], 1 + EPI_WARPS);  // the MMA thread and every epilogue warp
        }
        for (int a = 0; a < NACC; ++a) {
            mbar_init(&tfull_bar[a], 1);
            mbar_init(&tempty_bar[a], 4);  // one arrival per epilogue warp of the tile's part
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.a128)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.b128)) : "memory");
        if constexpr (!CORR_EPI) {  // the tail boxes (8-bit)
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.a32)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.b32)) : "memory");
        }
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_s;

    if constexpr (!BATCH) grid_dep_sync();  // the operand rows, statistics and counts are written
    int *err0 = ctx[0].b.err;

    // items per slice: row tiles of the kept ranges x active candidate
    // splits (rows are the ranges kept for screening, columns the candidates
    // of the kept domains, both compacted in original order)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const SliceCtx &c = ctx[i];
        const int nrow = c.b.cb.counts[0], ncol = 8 * c.b.cb.counts[2];
        const int rt = (nrow + BM - 1) / BM, tiles = (ncol + SUPER - 1) / SUPER;
        const int ns = rt > 0 && tiles > 0 ? active_splits(rt, tiles, c.target, c.n_split, SUPER, c.g.m) : 0;
        ns_s[i] = ns;
        rt_s[i] = rt;
        ip_s[i + 1] = rt * ns;
    }
    __syncthreads();
    if (warp == 0) {  // inclusive scan of the item counts, 32 slices at a time
        int carry = 0;
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            int v = i < n ? ip_s[i + 1] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            if (i < n) ip_s[i + 1] = carry + v;
            carry += __shfl_sync(0xffffffffu, v, 31);
        }
        if (lane == 0) ip_s[0] = 0;
    }
    if (threadIdx.x == 0) {
        // self-check: every TMA box and MMA operand lies inside this CTA's
        // dynamic shared memory, and the TMEM allocation is lane field 0,
        // columns [base, base + TMEM_COLS) within the 512 of the SM
        const uint32_t used = (uint32_t)(smem - smem_raw) + A_BYTES + NSTG * B_BYTES + 32 * ET * 4 +
                              EPI_WARPS * DC_WARP * (16 + 4 + 32);
        int bad = 0;
        if (used > smem_bytes) bad = 2;
        if (smem_u32(smem) & 1023u) bad = 4;
        if ((tmem_base >> 16) != 0 || (tmem_base & 0xFFFFu) + TMEM_COLS > 512) bad = 5;
        abort_s = bad;
        if (bad) atomicExch(err0, bad);
    }
    __syncthreads();
    const int total = ip_s[n];
    if ((int)blockIdx.x >= total) {  // CTA-uniform: no work
        if (warp == 1) {
            __syncwarp();
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                         : "memory");
        }
        return;
    }
    const bool run = abort_s == 0;

    if (!run) {
        // skip all work; fall through to the TMEM release
    } else if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t bseq = 0;  // B tiles issued by this CTA
            int kitem = 0;      // items started
            bool a_pending = false;
            // items are taken from a queue shared by all CTAs (`queue`, a
            // counter zeroed by the statistics kernel) and handed to the other
            // roles in order
            for (int k = 0;; ++k) {
                const int slot = k % kItemQ;
                if (!mbar_wait(&q_empty[slot], ((k / kItemQ) & 1) ^ 1, &abort_s, err0, wait_ns)) break;
                // the first item of CTA b is item b (every CTA takes one), the
                // later ones come from the counter: items gridDim.x, gridDim.x + 1, ...
                int item = k == 0 ? (int)blockIdx.x : (int)gridDim.x + atomicAdd(queue, 1);
                if (item >= total || *(volatile int *)&abort_s) item = -1;
                item_q[slot] = item;
                mbar_arrive(&q_full[slot]);
                if (item < 0) break;
                const TcItem w = tc_item(ctx, ip_s, ns_s, rt_s, n, item);
                const SliceCtx &c = ctx[w.s];
                int *err = c.b.err;
                const int rpad = (c.g.R + BM - 1) / BM * BM, npad = (c.g.N + SUPER - 1) / SUPER * SUPER;
                if (w.r0 + BM > rpad || w.t_end * SUPER > npad) {  // every box inside the slice's padded operands
                    abort_s = 3;
                    atomicExch(err, 3);
                    break;
                }
                // the previous item's MMAs must be done with A
                if (kitem > 0 && !mbar_wait(&a_empty, (kitem - 1) & 1, &abort_s, err, wait_ns)) break;
                mbar_expect_tx(&a_full, A_TX);
                if constexpr (KB == 1 && PARTS == 2) {
                    tma_load_2d(sA, &maps.a128, 0, c.abase + w.r0, &a_full);
                } else if constexpr (KB == 1) {
#pragma unroll
                    for (int b = 0; b < NBLK; ++b)
                        tma_load_2d(sA + b * A_BLK, &maps.a128, BW * b, c.abase + w.r0, &a_full);
                    tma_load_2d(sA + NBLK * A_BLK, &maps.a32, BW * NBLK, c.abase + w.r0, &a_full);
                } else {
#pragma unroll
                    for (int b = 0; b < KB; ++b) tma_load_2d(sA + b * A_BLK, &maps.a128, BW * b, c.abase + w.r0, &a_full);
                }
                a_pending = true;
                ++kitem;
                bool ok = true;
                for (int t = w.t_begin * LISTS; ok && t < w.t_end * LISTS; ++t) {  // MMA tiles of the item
                    const int y = c.bbase + t * BN;
                    if constexpr (KB == 1) {
                        const int s = bseq % NSTG;
                        if (!(ok = mbar_wait(&empty_bar[s], ((bseq / NSTG) & 1) ^ 1, &abort_s, err, wait_ns))) break;
                        uint8_t *dst = sB + s * B_BYTES;
                        mbar_expect_tx(&full_bar[s], B_TX);
#pragma unroll
                        for (int b = 0; b < NBLK; ++b) tma_load_2d(dst + b * B_BLK, &maps.b128, BW * b, y, &full_bar[s]);
                        if constexpr (!CORR_EPI) tma_load_2d(dst + NBLK * B_BLK, &maps.b32, BW * NBLK, y, &full_bar[s]);
                        ++bseq;
                    } else {
                        // part p, box b: columns 64 (p KB + b) of the candidate rows
                        for (int pb = 0; pb < NBLK * KB; ++pb) {
                            const int s = bseq % NSTG;
                            if (!(ok = mbar_wait(&empty_bar[s], ((bseq / NSTG) & 1) ^ 1, &abort_s, err, wait_ns)))
                                break;
                            mbar_expect_tx(&full_bar[s], B_TX);
                            tma_load_2d(sB + s * B_BYTES, &maps.b128, BW * pb, y, &full_bar[s]);
                            ++bseq;
                        }
                    }
                }
                if (!ok) break;
            }
            // drain: every issued load must land before the CTA may exit
            if (a_pending && !mbar_try_wait(&a_full, (kitem - 1) & 1)) {
                const unsigned long long t0 = gtimer();
                while (!mbar_try_wait(&a_full, (kitem - 1) & 1) && gtimer() - t0 < kDrainNs) {
                }
            }
            for (uint32_t q = (bseq > NSTG ? bseq - NSTG : 0); q < bseq; ++q) {
                const int s = q % NSTG;
                if (mbar_try_wait(&full_bar[s], (q / NSTG) & 1)) continue;
                const unsigned long long t0 = gtimer();
                while (!mbar_try_wait(&full_bar[s], (q / NSTG) & 1) && gtimer() - t0 < kDrainNs) {
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t a_base = smem_u32(sA);
            const uint32_t b_base0 = smem_u32(sB);
            uint32_t bseq = 0, aseq = 0;
            uint64_t *last_bar = nullptr;  // the barrier of the last commit, and its phase parity
            uint32_t last_par = 0;
            int kitem = 0;
            bool ok = true;
            for (int k = 0; ok; ++k) {
                const int slot = k % kItemQ;
                if (!(ok = mbar_wait(&q_full[slot], (k / kItemQ) & 1, &abort_s, err0, wait_ns))) break;
                const int item = item_q[slot];
                mbar_arrive(&q_empty[slot]);
                if (item < 0) break;
                const TcItem w = tc_item(ctx, ip_s, ns_s, rt_s, n, item);
                int *err = ctx[w.s].b.err;
                if (!(ok = mbar_wait(&a_full, kitem & 1, &abort_s, err, wait_ns))) break;
                ++kitem;
                for (int t = w.t_begin * LISTS; t < w.t_end * LISTS; ++t, ++aseq) {  // MMA tiles, in order
                    const int acc = aseq % NACC;
                    if (!(ok = mbar_wait(&tempty_bar[acc], ((aseq / NACC) & 1) ^ 1, &abort_s, err, wait_ns))) break;
                    const uint32_t d_tmem = tmem_base + acc * ACC_COLS;
                    if constexpr (KB == 1) {
                        const int s = bseq % NSTG;
                        if (!(ok = mbar_wait(&full_bar[s], (bseq / NSTG) & 1, &abort_s, err, wait_ns))) break;
                        tc_fence_after();
                        const uint32_t b_base = b_base0 + s * B_BYTES;
                        if constexpr (PARTS == 2) {
                            // The stage's hi block (candidate rows 0..BN-1) and lo block (the same
                            // candidates' lo parts, rows BN..2BN-1) lie one after the other in whole
                            // 8-row groups, so they are one operand of 2 BN rows against the range
                            // pixels (A block 0): one MMA per K step puts hi in slot columns [0, BN)
                            // and lo in [BN, 2 BN), half the MMA instructions of a pair per block.
#pragma unroll
                            for (int sub = 0; sub < KPB; ++sub)
                                umma_f16(d_tmem, smem_desc(a_base + sub * 32, SBO, LAYOUT),
                                         smem_desc(b_base + sub * 32, SBO, LAYOUT), IDESC2, sub ? 1u : 0u);
                        } else {
                            // 8-bit: the q' block, then the tail block with the centring terms
#pragma unroll
                            for (int k = 0; k < KSTEPS; ++k) {
                                const bool tail = k == NBLK * KPB;
                                const int blk = k / KPB, sub = k % KPB;
                                const uint64_t ad = tail ? smem_desc(a_base + NBLK * A_BLK, 256, 6)
                                                         : smem_desc(a_base + blk * A_BLK + sub * 32, SBO, LAYOUT);
                                const uint64_t bd = tail ? smem_desc(b_base + NBLK * B_BLK, 256, 6)
                                                         : smem_desc(b_base + blk * B_BLK + sub * 32, SBO, LAYOUT);
                                umma_f16(d_tmem, ad, bd, IDESC, k > 0 ? 1u : 0u);
                            }
                        }
                        umma_commit(&empty_bar[s]);  // smem stage free once these MMAs finish
                        ++bseq;
                    } else {
                        // part p accumulates its KB boxes (K = 64 each) into
                        // columns [p BN, (p + 1) BN) of the slot
                        for (int pb = 0; pb < NBLK * KB; ++pb) {
                            const int s = bseq % NSTG;
                            if (!(ok = mbar_wait(&full_bar[s], (bseq / NSTG) & 1, &abort_s, err, wait_ns))) break;
                            tc_fence_after();
                            const int p = pb / KB, b = pb % KB;
                            const uint32_t b_base = b_base0 + s * B_BYTES;
#pragma unroll
                            for (int sub = 0; sub < KPB; ++sub)
                                umma_f16(d_tmem + p * BN, smem_desc(a_base + b * A_BLK + sub * 32, SBO, LAYOUT),
                                         smem_desc(b_base + sub * 32, SBO, LAYOUT), IDESC, (b | sub) ? 1u : 0u);
                            umma_commit(&empty_bar[s]);
                            last_bar = &empty_bar[s];
                            last_par = (bseq / NSTG) & 1;
                            ++bseq;
                        }
                        if (!ok) break;
                    }
                    umma_commit(&tfull_bar[acc]);  // accumulator ready for the epilogue
                    last_bar = &tfull_bar[acc];
                    last_par = (aseq / NACC) & 1;
                }
                if (!ok) break;
                umma_commit(&a_empty);  // A free once the item's MMAs finish
            }
            // drain: the MMAs issued so far must finish before the CTA frees
            // TMEM and shared memory (after an abort the epilogue no longer
            // waits for them); the last commit tracks all of them
            if (last_bar && !mbar_try_wait(last_bar, last_par)) {
                const unsigned long long t0 = gtimer();
                while (!mbar_try_wait(last_bar, last_par) && gtimer() - t0 < kDrainNs) {
                }
            }
        }
    } else {
        // ------------------------------------------------------ epilogue
        const int ew = warp - 2;              // epilogue warp 0..EPI_WARPS-1
        const int quad = warp & 3;            // TMEM lane quadrant this warp may access
        const int part = ew >> 2;             // which 32 columns of each tile
        const int row = quad * 32 + lane;
        const int et = ew * 32 + lane;        // staging column of this thread
        float4 *wdc = dcs + ew * DC_WARP;
        int *wod = reinterpret_cast<int *>(dcs + EPI_WARPS * DC_WARP) + ew * DC_WARP;
        DcPack *wdp = dps + ew * DC_WARP;
        const uint32_t lane_addr = tmem_base + ((uint32_t)(quad * 32) << 16);
        uint32_t aseq = 0;
        bool ok = true;
        for (int k = 0; ok; ++k) {
            const int slot = k % kItemQ;
            if (!(ok = __all_sync(0xffffffffu, mbar_wait(&q_full[slot], (k / kItemQ) & 1, &abort_s, err0, wait_ns)))) break;
            const int item = item_q[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&q_empty[slot]);
            if (item < 0) break;
            const TcItem w = tc_item(ctx, ip_s, ns_s, rt_s, n, item);
            const SliceCtx &c = BATCH ? many[w.s] : one;
            const Geometry &g = c.g;
            // the slice's constants: kernel parameters (constant-bank operands) for
            // a single search, the context array (cached loads) for a batch
            const EpiConst &ec = c.ec;
            const float4 *dconst = c.b.cb.dconst_c;
            const int *dmap = c.b.cb.dmap;
            int *err = c.b.err;
            int *tbest = c.b.tbest;
            const int nrow = c.b.cb.counts[0], ndom = c.b.cb.counts[2], ncol = 8 * ndom;
            const int jrow = w.r0 + row;          // search row
            const bool live = jrow < nrow;
            const int r = live ? c.b.cb.act[jrow] : 0;  // range id
            RangeEpi re{};
            if (live) re = range_epi(c.b.ri[r], ec);
            const float er = (CORR_EPI && live) ? (float)c.b.ri[r].e_r : 0.0f;  // centring correction factor
            const f32x2_t er2 = pk2(er, er);
            const bool scr = live && (dense || !re.shadow);
            // the key every s-code-0 candidate of this range gets (one value:
            // with c = 0 the key is lambda * w^2 of the offset residue of zb)
            const float K0 = epi_key(0.0f, 0.0f, 0.0f, re.zb, make_float4(0.f, 0.f, 0.f, 0.f), ec);
            ListState L;
            list_init(L);
            const int ntile = w.t_end - w.t_begin;  // super-tiles of the item
            // prefetch for the first chunk: its 4 domains and the shared best key
            float4 dc_next = make_float4(0.f, 0.f, 0.f, 0.f);
            int od_next = 0;
            int tb_next = 0x7f800000;
            if (ntile > 0) {
                const int jd = ((w.t_begin * SUPER + part * BN) >> 3) + lane;
                if (lane < DC_WARP && jd < ndom) {
                    dc_next = __ldg(dconst + jd);
                    od_next = __ldg(dmap + jd);
                }
                if (scr && !dump) tb_next = __ldcg(tbest + r);
            }
            for (int it = 0; ok && it < ntile; ++it) {
                // this part's MMA tile of super-tile it: the item's MMA tile 3 it + part
                const uint32_t mt = aseq + it * LISTS + part;
                const int acc = mt % NACC;
                if (scr && !dump) {
                    const float Tg = ord2f(tb_next);  // best key other CTAs found
                    list_adopt(L, Tg, re, ec);
                    L.Tpub = fminf(L.Tpub, Tg);
                }
                // warp-uniform decision: tcgen05.ld below is .sync.aligned
                if (!(ok = __all_sync(0xffffffffu, mbar_wait(&tfull_bar[acc], (mt / NACC) & 1, &abort_s, err, wait_ns))))
                    break;
                tc_fence_after();
#pragma unroll 1
                for (int ch = 0; ch < CHUNKS; ++ch) {
                    const int n0 = (w.t_begin + it) * SUPER + part * BN + ch * EPI_COLS;
                    __syncwarp();  // every lane is done with the previous chunk's staged constants
                    if (lane < DC_WARP) {
                        wdc[lane] = dc_next;
                        wod[lane] = od_next;
                        wdp[lane] = dc_pack(dc_next, ec);
                    }
                    {  // prefetch for the next chunk: the tile's second, or the next super-tile's first
                        const int n1 = ch + 1 < CHUNKS ? n0 + EPI_COLS : n0 + SUPER - (CHUNKS - 1) * EPI_COLS;
                        const bool more = ch + 1 < CHUNKS || it + 1 < ntile;
                        const int jd = (n1 >> 3) + lane;
                        if (more && lane < DC_WARP && jd < ndom) {
                            dc_next = __ldg(dconst + jd);
                            od_next = __ldg(dmap + jd);
                        }
                        if (ch + 1 == CHUNKS && it + 1 < ntile && scr && !dump) tb_next = __ldcg(tbest + r);
                    }
                    __syncwarp();
                    const uint32_t taddr = lane_addr + acc * ACC_COLS + ch * EPI_COLS;
                    const int nv = min(32, ncol - n0);  // may be <= 0 in the last tile
                    // the chunk's domain constants stay in shared memory (read where
                    // used, which leaves the registers to the key computation)
                    const int (&od)[4] = *reinterpret_cast<const int (*)[4]>(wod);
                    const float4 (&dc)[4] = *reinterpret_cast<const float4 (*)[4]>(wdc);
                    float X[32];
                    {
                        uint32_t h[32], l[32];
                        tmem_ld32(taddr, h);
                        if (PARTS == 2) {
                            tmem_ld32(taddr + BN, l);
                            tmem_wait2(h, l);
#pragma unroll
                            for (int j = 0; j < 32; j += 2)
                                upk2(add2(pk2(__uint_as_float(h[j]), __uint_as_float(h[j + 1])),
                                          pk2(__uint_as_float(l[j]), __uint_as_float(l[j + 1]))), X[j], X[j + 1]);
                        } else {
                            tmem_wait(h);
#pragma unroll
                            for (int j = 0; j < 32; ++j) X[j] = __uint_as_float(h[j]);
                        }
                    }
                    if (ch + 1 == CHUNKS) {
                        // the tile's accumulator is in registers: release it to the
                        // MMA warp now, so that a slow warp holds up the tensor
                        // cores only by its loads
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&tempty_bar[acc]);
                    }
                    if (dump) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float ca = CORR_EPI ? epi_corr(er, pick4(dc, j >> 3).w, ec) : 0.0f;
                            if (live && j < nv) dump[(size_t)r * g.N + od[j >> 3] * 8 + (j & 7)] = X[j] + ca;
                        }
                    } else {
                        if (nv < 32) {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (j >= nv) X[j] = __int_as_float(0x7fc00000);  // NaN: never listed
                        }
                        const float thr = fminf(L.key[kListK - 1], L.tw);
                        // s-code-0 candidates need the penalty only where one is
                        // listed already and their common key K0 is below the
                        // threshold (rare): the warp takes the plain keys otherwise
                        const bool zero_pen = __any_sync(0xffffffffu, scr && L.has_zero && K0 < thr);
                        uint32_t mask = 0u;
                        if (zero_pen)
                            mask = epi_keys32_tc<true>(X, wdp, re.zb, re.rho_lim, er2, ec, thr,
                                                       L.has_zero ? kZeroPenalty : 0.0f);
                        else
                            mask = epi_keys32_tc<false>(X, wdp, re.zb, re.rho_lim, er2, ec, thr, 0.0f);
                        mask = scr && nv > 0 ? mask & col_mask(nv) : 0u;
                        if (__any_sync(0xffffffffu, mask != 0u))
                            rare_chunk(X, mask, od, dc, er, xsm + et, ET, re, ec, L, tbest + r);
                    }
                }
            }
            aseq += ntile * LISTS;
            if (ok && scr && !dump) {
                ListEntry *dst = c.b.lists + (((size_t)r * c.n_split + w.split) * LISTS + part) * kListK;
#pragma unroll
                for (int i = 0; i < kListK; ++i) dst[i] = ListEntry{L.key[i], L.idx[i]};
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

// One search (one = its slice context, many = nullptr) or a batch of n
// slices (many: device array) whose operands share the tensor maps' buffers
// (rows from abase / bbase on); one CTA per SM, persistent.
template <int NBLK, int BW, int KB, bool BATCH>
__global__ void __launch_bounds__(THREADS, 1)
    k_search_tc(const __grid_constant__ TcMaps maps, const __grid_constant__ SliceCtx one, const SliceCtx *many, int n,
                int dense, float *dump, uint32_t smem_bytes, int *queue, unsigned long long wait_ns)
{
    search_tc_run<NBLK, BW, KB, BATCH>(maps, one, many, n, dense, dump, smem_bytes, queue, wait_ns);
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map(CUtensorMap *m, const void *base, int rows, int kp, int x_box, int y_box, CUtensorMapSwizzle sw)
{
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)x_box, (cuuint32_t)y_box};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// K elements of one TMA box of pixels: m = 64 (n = 8) and m = 256 (n = 16,
// four boxes per copy of the pixels) in 128B-swizzled boxes of 64, m = 16
// (n = 4) in 32B-swizzled ones.
static int tc_block_width(const Geometry &g) { return g.m == 64 || g.m == 256 ? 64 : (g.m == 16 ? 16 : 0); }

bool search_tc_supported(const Geometry &g)
{
    const int bw = tc_block_width(g);
    return bw != 0 && g.KP == (g.split_hilo ? 2 : 1) * g.m + 16;
}

size_t search_tc_smem(const Geometry &g)
{
    const int nblk = g.split_hilo ? 2 : 1, bw = tc_block_width(g);
    const size_t epi = 32 * (32 * EPI_WARPS) * 4 + EPI_WARPS * DC_WARP * (16 + 4 + 32);
    if (g.m == 256)  // the range pixels once (4 boxes), a ring of 7 one-box stages
        return 1024 + (size_t)4 * BM * bw * 2 + (size_t)7 * BN * bw * 2 + epi;
    return 1024 + (size_t)(nblk * BM * bw * 2 + BM * 32) + (size_t)STAGES * (nblk * BN * bw * 2 + BN * 32) + epi;
}

int search_tc_lists_per_split() { return LISTS; }

int search_tc_tile() { return SUPER; }

int search_tc_rows(int rows) { return (rows + BM - 1) / BM * BM; }

int search_tc_cols(int cols) { return (cols + SUPER - 1) / SUPER * SUPER; }

// Limit of the search's pipeline waits (fic_set_wait_limit_ns), read at
// each launch.
static std::atomic<unsigned long long> g_wait_ns{kDefaultWaitNs};

unsigned long long wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

void set_wait_limit_ns(unsigned long long ns) { g_wait_ns.store(ns ? ns : kDefaultWaitNs, std::memory_order_relaxed); }

static int n_sms()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <int NBLK, int BW, int KB, bool BATCH>
static cudaError_t launch_tc3(const TcMaps &mp, const SliceCtx &one, const SliceCtx *many, int n, int dense,
                              float *dump, int *queue, size_t smem, cudaStream_t st)
{
    cudaError_t e =
        cudaFuncSetAttribute(k_search_tc<NBLK, BW, KB, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_dep(k_search_tc<NBLK, BW, KB, BATCH>, dim3(n_sms()), dim3(THREADS), smem, st, mp, one, many, n,
                      dense, dump, (uint32_t)smem, queue, (unsigned long long)wait_limit_ns());
}

template <int NBLK, int BW, int KB>
static cudaError_t launch_tc(const TcMaps &mp, const SliceCtx &one, const SliceCtx *many, int n, int dense, float *dump,
                             int *queue, size_t smem, cudaStream_t st)
{
    return many ? launch_tc3<NBLK, BW, KB, true>(mp, one, many, n, dense, dump, queue, smem, st)
                : launch_tc3<NBLK, BW, KB, false>(mp, one, many, n, dense, dump, queue, smem, st);
}

// Tensor maps over an operand pair (arows / brows rows of KP halves) and
// the launch; g: the geometry of any of the slices (pixel and code layout).
static cudaError_t launch_tc_any(const Geometry &g, const __half *ra16, int arows, const __half *cb16, int brows,
                                 const SliceCtx &one, const SliceCtx *many, int n, int dense, float *dump,
                                 int *queue, cudaStream_t st)
{
    if (!search_tc_supported(g) || n < 1 || n > kMaxBatch || !queue) return cudaErrorInvalidValue;
    if (!many && n != 1) return cudaErrorInvalidValue;  // the single-search kernel sizes its tables for one slice
    TcMaps mp;
    const int nblk = g.split_hilo ? 2 : 1, bw = tc_block_width(g);
    const CUtensorMapSwizzle sw = bw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B;
    if (!make_map(&mp.a128, ra16, arows, g.KP, bw, BM, sw) ||
        !make_map(&mp.a32, ra16, arows, g.KP, 16, BM, CU_TENSOR_MAP_SWIZZLE_32B) ||
        !make_map(&mp.b128, cb16, brows, g.KP, bw, BN, sw) ||
        !make_map(&mp.b32, cb16, brows, g.KP, 16, BN, CU_TENSOR_MAP_SWIZZLE_32B))
        return cudaErrorInvalidValue;
    const size_t smem = search_tc_smem(g);
    if (g.m == 256)
        return nblk == 2 ? launch_tc<2, 64, 4>(mp, one, many, n, dense, dump, queue, smem, st)
                         : launch_tc<1, 64, 4>(mp, one, many, n, dense, dump, queue, smem, st);
    if (bw == 64)
        return nblk == 2 ? launch_tc<2, 64, 1>(mp, one, many, n, dense, dump, queue, smem, st)
                         : launch_tc<1, 64, 1>(mp, one, many, n, dense, dump, queue, smem, st);
    return nblk == 2 ? launch_tc<2, 16, 1>(mp, one, many, n, dense, dump, queue, smem, st)
                     : launch_tc<1, 16, 1>(mp, one, many, n, dense, dump, queue, smem, st);
}

cudaError_t launch_search_tc(const Geometry &g, const EpiConst &ec, const RangeInfo *ri, const CompactBufs &cb,
                             int dense, const __half *ra16, const __half *cb16, ListEntry *lists, int max_split,
                             int target, int *tbest, float *dump, int *err, int *queue, cudaStream_t st)
{
    SliceCtx one = {};
    one.g = g;
    one.ec = ec;
    one.b.ri = const_cast<RangeInfo *>(ri);
    one.b.cb = cb;
    one.b.lists = lists;
    one.b.tbest = tbest;
    one.b.err = err;
    one.n_split = max_split;
    one.target = target;
    // operand buffers hold whole boxes (rows padded to the box heights)
    return launch_tc_any(g, ra16, search_tc_rows(g.R), cb16, search_tc_cols(g.N), one, nullptr, 1, dense, dump, queue,
                         st);
}

cudaError_t launch_search_tc_batch(const Geometry &g, const __half *ra16, int arows, const __half *cb16, int brows,
                                   const SliceCtx *ctx, int n, int dense, int *queue, cudaStream_t st)
{
    const SliceCtx none = {};
    return launch_tc_any(g, ra16, arows, cb16, brows, none, ctx, n, dense, nullptr, queue, st);
}

}  // namespace fic
