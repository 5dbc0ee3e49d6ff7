// Exact re-scoring of the screened candidates, certification, exact fallback,
// and map output.
//
// The screening epilogue ranks candidates in FP32.  Here each range's list
// entries whose key lies within 2*beta of the best key are re-scored exactly:
//   - the cross term X = sum q_i b_i is recomputed in integers,
//   - the s and o codes are decided in FP64 with the operation sequence of the
//     least squares of eq 9-12 (so they are identical to an FP64 evaluation of
//     the same formulas), and
//   - the residual of eq 8 is evaluated exactly in integer arithmetic:
//       R * D^2 = sum_i (c*Lo*q_i + 4*Ls*e*P - D*b_i)^2,  D = 4*Ls*Lo,
//     expanded into the exact integer statistics.
// The winner is the smallest exact residual, ties to the lowest candidate
// index (Algorithm 2's strict comparison).  A range is certified when every
// full candidate list's worst key lies beyond the re-scoring window, so no
// candidate outside the lists can beat or tie the winner; otherwise it goes
// to the exact fallback, which scans all of its candidates with exact
// integer decisions.
#include <algorithm>

#include "fic_internal.cuh"

namespace fic {

namespace {

struct Stats {
    long long Sq, Sqq, Sb, Sbb, X;
};

// FP64 least squares + quantisation, in the evaluation order of eq 9-12.
__device__ void fp64_codes(const Geometry &g, const Stats &st, int &c, int &e, double &s_hat,
                           double &o_hat)
{
    const double md = (double)g.m;
    const double Sa = __dmul_rn((double)st.Sq, 0.25);
    const double Sb = (double)st.Sb;
    const double Saa = __dmul_rn((double)st.Sqq, 0.0625);
    const double Sab = __dmul_rn((double)st.X, 0.25);
    const double den = __dsub_rn(__dmul_rn(md, Saa), __dmul_rn(Sa, Sa));
    const double s =
        (den == 0.0) ? 0.0 : __ddiv_rn(__dsub_rn(__dmul_rn(md, Sab), __dmul_rn(Sa, Sb)), den);
    const double Ls = (double)g.Ls;
    const double sc = s < -1.0 ? -1.0 : (s > 1.0 ? 1.0 : s);
    c = (int)round(__dmul_rn(sc, Ls));
    s_hat = __ddiv_rn((double)c, Ls);
    // m is a power of two: dividing by it is an exact scaling, the same
    // result as the multiplication by its exact reciprocal (off the chain)
    const double o = __dmul_rn(__dsub_rn(Sb, __dmul_rn(s_hat, Sa)), ldexp(1.0, -2 * g.ln));
    const double P = (double)g.P, Lo = (double)g.Lo;
    const double oc = o < -P ? -P : (o > P ? P : o);
    e = (int)round(__ddiv_rn(__dmul_rn(oc, Lo), P));
    o_hat = __ddiv_rn(__dmul_rn((double)e, P), Lo);
}

// The code decisions of fp64_codes without its chain of dependent FP64
// divisions (a long latency at the FP64 rate of this part).  s * Ls =
// 4 Ls (m X - Sq Sb) / (m Sqq - Sq^2) and o * Lo / P = (4 Ls Sb - c Sq) Lo /
// (4 Ls m P) are formed in FP32 from exact integers (relative error below
// 4 * 2^-24); fp64_codes forms the same values with numerator and
// denominator exact in FP64 and an error below 2^-49 * Lo.  Away from a
// rounding boundary both round to the same code; within 4e-7 * |value| +
// 1e-6 of one (a few in 10^5 candidates) this returns false and the caller
// takes fp64_codes itself, so the codes are those of the FP64 sequence bit
// for bit.  The clamps at +-Ls, +-Lo are integers, never boundaries.
__device__ __forceinline__ bool round_clear(float v, float lim, int &code)
{
    const float a = fminf(fabsf(v), lim);
    const float fl = floorf(a), fr = a - fl;  // exact
    if (fabsf(fr - 0.5f) <= fmaf(4e-7f, a, 1e-6f)) return false;
    const int k = (int)fl + (fr > 0.5f ? 1 : 0);
    code = v < 0.0f ? -k : k;
    return true;
}

__device__ __forceinline__ bool fast_codes(const Geometry &g, const Stats &st, int &c, int &e)
{
    const long long NI = (long long)g.m * st.X - st.Sq * st.Sb;
    const long long DI = (long long)g.m * st.Sqq - st.Sq * st.Sq;
    c = 0;
    if (DI != 0 && !round_clear(__fdiv_rn(__ll2float_rn(4LL * g.Ls * NI), __ll2float_rn(DI)), (float)g.Ls, c))
        return false;
    const long long NE = (4LL * g.Ls * st.Sb - (long long)c * st.Sq) * g.Lo;
    return round_clear(__fdiv_rn(__ll2float_rn(NE), __ll2float_rn(4LL * g.Ls * g.m * g.P)), (float)g.Lo, e);
}

// s_hat = c / Ls and o_hat = e P / Lo as floats: Ls and Lo are 2^k - 1, so
// a quotient of integers by them is exact or has a binary expansion of
// period k <= 9, which never holds the 28 equal bits after the float's last
// place that would make the double quotient a float rounding midpoint; the
// float rounding of the double quotient is then the correctly rounded float
// quotient (when the numerator is exact in FP32).
__device__ __forceinline__ float s_hat_f(const Geometry &g, int c)
{
    return __fdiv_rn((float)c, (float)g.Ls);
}

__device__ __forceinline__ float o_hat_f(const Geometry &g, int e)
{
    const long long eP = (long long)e * g.P;
    if (eP < (1LL << 24) && eP > -(1LL << 24)) return __fdiv_rn((float)eP, (float)g.Lo);
    return (float)__ddiv_rn((double)eP, (double)g.Lo);
}

// Exact integer arithmetic in one of two widths: 64-bit when every term of
// the residual expansion below stays under 2^62 (Geometry::wide == 0, checked
// on the host from the largest statistics the bit depth allows), 128-bit
// otherwise.
template <bool Wide> struct Exact;
template <> struct Exact<false> {
    typedef long long S;
    typedef unsigned long long U;
};
template <> struct Exact<true> {
    typedef __int128 S;
    typedef unsigned __int128 U;
};

// Exact residual times D^2 for codes (c, e).
template <bool Wide>
__device__ __forceinline__ typename Exact<Wide>::S exact_err(const Geometry &g, const Stats &st, int c, int e)
{
    typedef typename Exact<Wide>::S S;
    const S A = (S)c * g.Lo;
    const S Bo = (S)4 * g.Ls * e * g.P;
    const S Dd = (S)4 * g.Ls * g.Lo;
    return A * A * st.Sqq + (S)g.m * Bo * Bo + Dd * Dd * st.Sbb + 2 * A * Bo * st.Sq - 2 * A * Dd * st.X -
           2 * Bo * Dd * st.Sb;
}

template <typename U>
__device__ __forceinline__ bool better(U e1, uint32_t i1, U e2, uint32_t i2)
{
    return e1 < e2 || (e1 == e2 && i1 < i2);
}

__device__ __forceinline__ unsigned long long shfl_xor64(unsigned long long v, int off)
{
    return __shfl_xor_sync(0xffffffffu, v, off);
}

__device__ __forceinline__ unsigned __int128 shfl_xor128(unsigned __int128 v, int off)
{
    const unsigned long long lo = shfl_xor64((unsigned long long)v, off);
    const unsigned long long hi = shfl_xor64((unsigned long long)(v >> 64), off);
    return ((unsigned __int128)hi << 64) | lo;
}

__device__ __forceinline__ unsigned long long shfl_xor_u(unsigned long long v, int off) { return shfl_xor64(v, off); }
__device__ __forceinline__ unsigned __int128 shfl_xor_u(unsigned __int128 v, int off) { return shfl_xor128(v, off); }

// Warp argmin over (err, idx).
template <typename U>
__device__ __forceinline__ void warp_argmin(U &err, uint32_t &idx)
{
    for (int off = 16; off > 0; off >>= 1) {
        const U oe = shfl_xor_u(err, off);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, idx, off);
        if (better(oe, oi, err, idx)) {
            err = oe;
            idx = oi;
        }
    }
}

// Warp argmin over (err, idx) carrying the winner's cross term x.
template <typename U>
__device__ __forceinline__ void warp_argmin_x(U &err, uint32_t &idx, long long &x)
{
    for (int off = 16; off > 0; off >>= 1) {
        const U oe = shfl_xor_u(err, off);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, idx, off);
        const long long ox = __shfl_xor_sync(0xffffffffu, x, off);
        if (better(oe, oi, err, idx)) {
            err = oe;
            idx = oi;
            x = ox;
        }
    }
}

}  // namespace

// Cross-term word of a range whose winner's cross term the map output must
// compute itself (a range the search did not screen and that is not constant).
constexpr long long kNoCross = (long long)0x8000000000000000ull;

// The cross term of candidate 0 (domain 0, identity) for a range the search
// did not screen: for a constant range (pixel value Sb/m) it is Sb/m * Sq of
// domain 0; otherwise (a range the caller left out) unknown.
__device__ __forceinline__ long long unscreened_cross(const Geometry &g, const RangeInfo &rin, const DomainInfo *di)
{
    return rin.shadow ? (rin.Sb >> (2 * g.ln)) * di[0].Sq : kNoCross;
}

__device__ __forceinline__ double u128_to_double(unsigned __int128 v)
{
    return (double)(unsigned long long)(v >> 64) * 18446744073709551616.0 + (double)(unsigned long long)v;
}

// An FP32 value >= v (v an unsigned 128-bit integer below 2^127): the top 64
// significant bits, or-ed with 1 so that a discarded remainder always rounds
// the conversion up past them, converted upward and scaled exactly.
__device__ __forceinline__ float to_float_ru(unsigned __int128 v)
{
    const unsigned long long hi = (unsigned long long)(v >> 64);
    if (hi == 0) return __ull2float_ru((unsigned long long)v);
    const int sh = 64 - __clzll(hi);
    return ldexpf(__ull2float_ru((unsigned long long)(v >> sh) | 1ull), sh);
}

__device__ __forceinline__ float to_float_ru(unsigned long long v) { return __ull2float_ru(v); }

// round half away from zero of num/den (den > 0), exactly: an FP32 estimate
// corrected with exact integer comparisons.
__device__ __forceinline__ long long round_div_away(long long num, long long den)
{
    const long long a = num < 0 ? -num : num;
    long long q = (long long)(__fdividef((float)a, (float)den) + 0.5f);
    // want q = floor((2a + den) / (2 den))
    while (q > 0 && 2 * a + den < 2 * den * q) --q;
    while (2 * a + den >= 2 * den * (q + 1)) ++q;
    return num < 0 ? -q : q;
}

// Exact residual (times D^2) of candidate idx for range statistics st, with
// the s and o codes decided exactly from the rational least-squares values.
template <bool Wide>
__device__ __forceinline__ typename Exact<Wide>::U exact_rational(const Geometry &g, Stats st, const DomainInfo &dd,
                                                                 long long X)
{
    st.Sq = dd.Sq;
    st.Sqq = dd.Sqq;
    st.X = X;
    const long long den = (long long)g.m * dd.Sqq - dd.Sq * dd.Sq;
    const long long num = (long long)g.m * X - dd.Sq * st.Sb;
    int c = 0;
    if (den != 0) {
        const long long v = 4LL * num;  // s = v / den
        if (v >= den) c = g.Ls;
        else if (-v >= den) c = -g.Ls;
        else c = (int)round_div_away((long long)g.Ls * v, den);
    }
    const long long Q = 4LL * g.Ls * g.m * g.P;  // o * Lo / P = z * Lo / Q
    const long long z = 4LL * g.Ls * st.Sb - (long long)c * dd.Sq;
    int e = (int)round_div_away(z * g.Lo, Q);
    if (e > g.Lo) e = g.Lo;  // o is never below -P; clamp above only
    return (typename Exact<Wide>::U)exact_err<Wide>(g, st, c, e);
}

// Exact sum over the warp of q[j] * b[j] (lane l holds the terms of pixels
// l, l + 32, ...); every lane gets the sum.
__device__ __forceinline__ long long warp_dot(const int (&q)[kMaxM / 32], const int (&b)[kMaxM / 32])
{
    long long a = 0;
#pragma unroll
    for (int j = 0; j < kMaxM / 32; ++j) a += (long long)q[j] * b[j];
    for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
    return a;
}

// Finalists up to which the re-score takes them one at a time over the whole
// warp (latency of one gather each) rather than one per lane (staging of the
// permuted range pixels and a serial row per lane).
constexpr int kCoopFinalists = 4;

// The range's pixels permuted for each symmetry: bk[k*(m+1) + j] is the
// range pixel that S_k places over contracted-domain pixel j, so that
// X(d, k) = sum_j q_d[j] * bk[k][j] with the domain row read in natural order.
// Row pitch m+1 words: lanes of different symmetries hit different banks.
__device__ void stage_sym_pixels(const Geometry &g, const int (&b)[kMaxM / 32], int *bk)
{
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
#pragma unroll
        for (int j = 0; j < kMaxM / 32; ++j) {
            const int i = lane + 32 * j;
            if (i < g.m) {
                int sy, sx;
                sym_src(k, g.n, i >> g.ln, i & (g.n - 1), sy, sx);
                bk[k * (g.m + 1) + (sy << g.ln) + sx] = b[j];
            }
        }
    }
    __syncwarp();
}

// Exact X of candidate idx computed by one lane alone (16-byte loads of the
// domain row; m is a multiple of 16).
__device__ long long lane_cross(const Geometry &g, const uint16_t *qblk, uint32_t idx, const int *bk)
{
    const int *bkk = bk + (idx & 7) * (g.m + 1);
    const uint4 *qrow = reinterpret_cast<const uint4 *>(qblk + (size_t)(idx >> 3) * g.m);
    unsigned long long acc = 0;
#pragma unroll 4
    for (int v = 0; v < g.m / 8; ++v) {
        const uint4 w = __ldg(qrow + v);
        const int *bb = bkk + 8 * v;
        // eight products of at most 4P * P < 2^26 each: exact in 32 bits
        uint32_t s = (w.x & 0xffffu) * (uint32_t)bb[0] + (w.x >> 16) * (uint32_t)bb[1];
        s += (w.y & 0xffffu) * (uint32_t)bb[2] + (w.y >> 16) * (uint32_t)bb[3];
        s += (w.z & 0xffffu) * (uint32_t)bb[4] + (w.z >> 16) * (uint32_t)bb[5];
        s += (w.w & 0xffffu) * (uint32_t)bb[6] + (w.w >> 16) * (uint32_t)bb[7];
        acc += s;
    }
    return (long long)acc;
}

// One warp per range.  Ranking here uses exact integer arithmetic only
// (codes rounded exactly from the rational least-squares values, residual in
// 128-bit integers); the FP64 code decision of eq 9-12 is made once, for the
// winner, by k_finalize.  The two decisions differ only when an FP64
// rounding crosses a half-integer that the exact value misses by less than
// 1e-15 relative.
//  1. U = exact residual of the entry with the best screening key.
//  2. Finalists: entries whose key, less the screening error allowance,
//     does not exceed U (keys may underestimate, never overestimate by more
//     than the allowance).  The winner is the smallest exact residual, ties
//     to the lowest index.
//  3. Certified when every full list's last key, less the allowance at that
//     key, is strictly above the winner's residual: then no candidate outside
//     the lists can beat or tie it.  Otherwise the range goes to the exact
//     fallback.
// Both tests compare FP32 keys against thresholds computed once per range in
// FP64 and rounded outward (up for the finalist bound, so that no finalist
// is lost; the certification side is rounded down on the key and up on the
// threshold, so that it never certifies what the exact test would not).
struct Partial {
    unsigned long long lo, hi;
    uint32_t idx, pad;
};

// Re-scan of failed lists: work items (range << 7 | list), per (range, list)
// partial minima, per range the finalists' best and the items still pending.
struct SpanBufs {
    int *items;
    int *count;
    Partial *part;   // [R][max_lists]
    Partial *cert;   // [R]
    int *pending;    // [R]
};

__host__ __device__ SpanBufs span_bufs(const Geometry &g, int max_lists, void *ws, int *count)
{
    SpanBufs b;
    char *p = static_cast<char *>(ws);
    b.part = reinterpret_cast<Partial *>(p);
    p += sizeof(Partial) * (size_t)g.R * max_lists;
    b.cert = reinterpret_cast<Partial *>(p);
    p += sizeof(Partial) * (size_t)g.R;
    b.items = reinterpret_cast<int *>(p);
    p += sizeof(int) * (size_t)g.R * max_lists;
    b.pending = reinterpret_cast<int *>(p);
    b.count = count;
    return b;
}

size_t span_bytes(const Geometry &g, int max_lists)
{
    return (sizeof(Partial) + sizeof(int)) * (size_t)g.R * max_lists + (sizeof(Partial) + sizeof(int)) * (size_t)g.R;
}

__host__ __device__ inline int fallback_chunks(const Geometry &g) { return min(64, max(1, g.N / 1024)); }

// Partial results [R][chunks], then one completion counter per slot.
__host__ __device__ inline int *fallback_done(const Geometry &g, void *partial)
{
    return reinterpret_cast<int *>(reinterpret_cast<Partial *>(partial) + (size_t)g.R * fallback_chunks(g));
}

__device__ __forceinline__ unsigned long long hi64(unsigned long long) { return 0ull; }
__device__ __forceinline__ unsigned long long hi64(unsigned __int128 v) { return (unsigned long long)(v >> 64); }

// Winner words the re-score leaves for ranges whose winner an exact scan
// decides (never a resolved winner: those are index | 2^31 with index < 2^31 - 8).
constexpr uint32_t kWinScan = 0xffffffffu;   // queued for the full exact scan
constexpr uint32_t kWinLists = 0xfffffffeu;  // lists queued for exact re-scans
__device__ __forceinline__ bool win_pending(uint32_t w) { return w >= kWinLists; }

constexpr int kRescoreWarps = 4;
constexpr int kRescoreEnt = 16;  // list entries per lane: up to 512 per range
// Shared memory of a re-score warp: the symmetry-permuted range pixels
// (8 rows of m+1) and the finalist list (up to every entry).
__host__ __device__ constexpr int rescore_warp_ints(int m) { return 8 * (m + 1) + 32 * kRescoreEnt; }
template <bool Wide>
__device__ __forceinline__ void rescore_range(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                                              const DomainInfo *di, const uint16_t *bblk, const uint16_t *qblk,
                                              const ListEntry *lists, int max_lists, const int *counts,
                                              int lists_per_split, int col_tile, int target, int max_split,
                                              int exact_scan, uint32_t *winner, long long *winx, int *fb_list,
                                              int *fb_count, int r,
                                              int *bk, const SpanBufs &sb)
{
    typedef typename Exact<Wide>::U U;
    const int lane = threadIdx.x & 31;
    // lists actually written by the search (its split count follows the kept counts)
    const int n_lists = lists_per_split *
                        active_splits((counts[0] + 127) / 128, (8 * counts[2] + col_tile - 1) / col_tile, target, max_split,
                                      col_tile, g.m);
    const ListEntry *L = lists + (size_t)r * max_lists * kListK;
    const int nent = n_lists * kListK;
    // every entry of the range's lists in registers (entry lane + 32 s), the
    // pixels and statistics loaded alongside: one memory latency
    // (an entry naming no candidate counts as empty: lists a search left
    // unwritten after a timed-out wait may hold anything)
    ListEntry ent[kRescoreEnt];
#pragma unroll
    for (int q = 0; q < kRescoreEnt; ++q) {
        const int f = lane + 32 * q;
        ent[q] = f < nent ? L[f] : ListEntry{__int_as_float(0x7f800000), 0xffffffffu};
        if ((ent[q].idx & kIdxMask) >= (uint32_t)g.N) ent[q] = ListEntry{__int_as_float(0x7f800000), 0xffffffffu};
    }
    const RangeInfo rin = ri[r];
    int b[kMaxM / 32];
#pragma unroll
    for (int j = 0; j < kMaxM / 32; ++j) {
        const int i = lane + 32 * j;
        b[j] = i < g.m ? (int)bblk[(size_t)r * g.m + i] : 0;
    }
    // best key (ties to the lower index) and best clean key
    float kb = __int_as_float(0x7f800000), kc = __int_as_float(0x7f800000);
    uint32_t ib = 0xffffffffu;
#pragma unroll
    for (int q = 0; q < kRescoreEnt; ++q) {
        const ListEntry e = ent[q];
        if (e.idx == 0xffffffffu) continue;
        const uint32_t idx = e.idx & kIdxMask;
        if (e.key < kb || (e.key == kb && idx < ib)) {
            kb = e.key;
            ib = idx;
        }
        if ((e.idx & kCleanBit) && e.key < kc) kc = e.key;
    }
    for (int off = 16; off > 0; off >>= 1) {
        const float ok = __shfl_xor_sync(0xffffffffu, kb, off);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, ib, off);
        if (ok < kb || (ok == kb && oi < ib)) {
            kb = ok;
            ib = oi;
        }
        kc = fminf(kc, __shfl_xor_sync(0xffffffffu, kc, off));
    }
    if (ib == 0xffffffffu || exact_scan) {  // no candidate was listed (or asked): exact scan
        if (lane == 0) {
            winner[r] = kWinScan;
            fb_list[atomicAdd(fb_count, 1)] = r;
        }
        return;
    }
    // the best-key candidate's domain pixels, gathered through its symmetry
    // (lane l: those over range pixels l, l + 32, ...), and its domain's
    // statistics: loaded now, under the threshold work below, for its exact
    // cross term (it is nearly always the only finalist)
    int qb[kMaxM / 32];
    {
        const int d = ib >> 3;
        const SymFlags sf = sym_flags(ib & 7, g.n);
#pragma unroll
        for (int j = 0; j < kMaxM / 32; ++j) {
            const int i = lane + 32 * j;
            qb[j] = i < g.m ? (int)qblk[(size_t)d * g.m + sym_src_index(sf, g.ln, i >> g.ln, i & (g.n - 1))] : 0;
        }
    }
    const DomainInfo dib = di[ib >> 3];
    Stats st;
    st.Sb = rin.Sb;
    st.Sbb = rin.Sbb;
    const RangeEpi re = range_epi(rin, ec);
    U best_e = ~(U)0;
    uint32_t best_i = 0xffffffffu;
    long long best_x = 0;  // the cross term of best_i (for the map output)
    // Ub >= the best exact residual, rounded up; every threshold below is an
    // FP32 bound rounded outward.  A clean entry gives it without exact work:
    // its residual is at most sbbc + (key + beta(key)) / (2 Ls).  Otherwise
    // the best-key entry is re-scored exactly first.
    float Ub;
    if (kc < __int_as_float(0x7f800000)) {
        Ub = __fadd_ru(rin.sbbc, __fdiv_ru(__fadd_ru(kc, beta_key(re, kc, ec)), ec.two_ls));
    } else {
        best_x = warp_dot(qb, b);
        best_e = exact_rational<Wide>(g, st, dib, best_x);  // integer work, same on every lane
        best_i = ib;
        Ub = __fmul_ru(to_float_ru(best_e), ec.invD2_up);
    }
    // screening error allowance (the epilogue's), evaluated at the largest key
    // that can still matter
    const float kreach = __fmul_ru(__fsub_ru(Ub, rin.sbbc), ec.two_ls);
    const float beta_k = fmaxf(beta_key(re, kb, ec), beta_key(re, fmaxf(kb, kreach), ec));
    // finalist: sbbc + key/(2Ls) - beta/(2Ls) <= U  <=>  key <= (U - sbbc)*2Ls + beta
    const float kfin = __fadd_ru(kreach, beta_k);
    // Flat domains were not screened: all their candidates have s = 0 and the
    // same residual, so only the first of them, (first flat domain, k = 0), can
    // win; it is a finalist of every range.  With s = 0 its residual needs no
    // cross term.
    const int dflat = counts[3];
    if (lane == 0 && dflat >= 0) {
        const long long Q = 4LL * g.Ls * g.m * g.P;
        int e0 = (int)round_div_away(4LL * g.Ls * st.Sb * g.Lo, Q);
        if (e0 > g.Lo) e0 = g.Lo;
        Stats s0 = st;
        s0.Sq = s0.Sqq = s0.X = 0;  // multiplied by c = 0
        const U fe = (U)exact_err<Wide>(g, s0, 0, e0);
        const uint32_t fi = (uint32_t)dflat * 8;
        if (better(fe, fi, best_e, best_i)) {
            best_e = fe;
            best_i = fi;
            best_x = 0;  // unused: with s = 0 the cross term drops out
        }
    }
    // finalists (entries whose key can still reach the best, but the best
    // itself), compacted into this warp's list in shared memory, then
    // re-scored one per lane in a single pass: per-lane exact cross terms
    // against the symmetry-permuted range pixels, exact rational codes
    int *fl = bk + 8 * (g.m + 1);
    int nfin = 0;
    __syncwarp();  // the list and bk of the warp's previous range are read
#pragma unroll
    for (int q = 0; q < kRescoreEnt; ++q) {
        const bool fin = ent[q].idx != 0xffffffffu && (ent[q].idx & kIdxMask) != best_i && ent[q].key <= kfin;
        const unsigned bal = __ballot_sync(0xffffffffu, fin);
        if (fin) fl[nfin + __popc(bal & ((1u << lane) - 1u))] = (int)(ent[q].idx & kIdxMask);
        nfin += __popc(bal);
    }
    if (nfin > 0 && nfin <= kCoopFinalists) {  // warp-uniform: the usual case
        // each finalist's cross term over the whole warp (gathered pixels,
        // shuffle sum), the best-key candidate's from the loads made above
        __syncwarp();
        for (int f = 0; f < nfin; ++f) {
            const uint32_t idx = (uint32_t)fl[f];
            long long X;
            DomainInfo dd;
            if (idx == ib) {
                X = warp_dot(qb, b);
                dd = dib;
            } else {
                const int d = idx >> 3;
                const SymFlags sf = sym_flags(idx & 7, g.n);
                int qf[kMaxM / 32];
#pragma unroll
                for (int j = 0; j < kMaxM / 32; ++j) {
                    const int i = lane + 32 * j;
                    qf[j] = i < g.m ? (int)qblk[(size_t)d * g.m + sym_src_index(sf, g.ln, i >> g.ln, i & (g.n - 1))]
                                    : 0;
                }
                dd = di[d];
                X = warp_dot(qf, b);
            }
            const U er = exact_rational<Wide>(g, st, dd, X);  // same on every lane
            if (better(er, idx, best_e, best_i)) {
                best_e = er;
                best_i = idx;
                best_x = X;
            }
        }
    } else if (nfin > 0) {  // many finalists: one per lane
        stage_sym_pixels(g, b, bk);
        __syncwarp();
        for (int f = lane; f < nfin; f += 32) {
            const uint32_t idx = (uint32_t)fl[f];
            const long long X = lane_cross(g, qblk, idx, bk);
            const U er = exact_rational<Wide>(g, st, di[idx >> 3], X);
            if (better(er, idx, best_e, best_i)) {
                best_e = er;
                best_i = idx;
                best_x = X;
            }
        }
    }
    warp_argmin_x(best_e, best_i, best_x);
    // certified list: sbbc + (last - beta(last))/(2Ls) > E*, tested as
    // round-down(last - beta) > round-up((E* - sbbc) * 2Ls).  A full list's
    // unlisted candidates have residual >= its last key less the allowance at
    // that key; that bound must clear the winner strictly.  Entry f is the
    // last of its list when f % 4 == 3 (lanes 3, 7, ...).
    const float Estar = __fmul_ru(to_float_ru(best_e), ec.invD2_up);
    const float kcert = __fmul_ru(__fsub_ru(Estar, rin.sbbc), ec.two_ls);
    // a list that fails the test is re-scanned exactly over its own candidates
    // (the columns the search gave it); the winner is then the best of those
    // scans and of the finalists above
    // The last entries sit on lanes 3, 7, ..., 31 (8 of them for each q); each
    // lane takes those of 4 values of q, gathered by shuffles, so that all 32
    // lanes test 4 lists instead of 8 lanes testing 16.  Lane l tests, for
    // q = l/8 + 4t, the list (l % 8) + 8q held by lane 4 (l % 8) + 3.
    static_assert(kListK == 4 && kRescoreEnt == 16, "certification: 8 list ends per entry row, 4 rows a lane");
    uint32_t failing = 0;  // bit q: list (lane % 8) + 8q failed
    {
        const int src = 4 * (lane & 7) + kListK - 1, q0 = lane >> 3;
        float lk[4];
        uint32_t li[4];
#pragma unroll
        for (int q = 0; q < kRescoreEnt; ++q) {
            const float k = __shfl_sync(0xffffffffu, ent[q].key, src);
            const uint32_t i = __shfl_sync(0xffffffffu, ent[q].idx, src);
            if ((q & 3) == q0) {
                lk[q >> 2] = k;
                li[q >> 2] = i;
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (li[t] == 0xffffffffu) continue;  // list not full (or past the end)
            if (!(__fsub_rd(lk[t], beta_key(re, lk[t], ec)) > kcert)) failing |= 1u << (q0 + 4 * t);
        }
    }
    int nfail = __popc(failing);
    for (int off = 16; off > 0; off >>= 1) nfail += __shfl_xor_sync(0xffffffffu, nfail, off);
    if (nfail == 0) {
        if (lane == 0) {
            winner[r] = best_i;
            winx[r] = best_x;
        }
        return;
    }
    Partial *sp = sb.part + (size_t)r * max_lists;
    for (int l = lane; l < n_lists; l += 32) sp[l] = Partial{~0ull, ~0ull, 0xffffffffu, 0};
    if (lane == 0) {
        sb.cert[r] = Partial{(unsigned long long)best_e, hi64(best_e), best_i, 0};
        sb.pending[r] = nfail;
        winner[r] = kWinLists;  // the last list scan writes the winner
    }
    while (failing) {
        const int q = __ffs(failing) - 1;
        failing &= failing - 1;
        const int l = (lane & 7) + 8 * q;
        sb.items[atomicAdd(sb.count, 1)] = (r << 7) | l;
    }
}

// Persistent warps over the screened ranges (act[], one warp per range, the
// grid sized to be resident at once); every other range is a constant one:
// num = 0 for every candidate, so s = 0, one offset and one residual for
// all, and the first candidate wins (Algorithm 2).
template <bool Wide>
__device__ __forceinline__ void rescore_blocks(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                                               const DomainInfo *di, const uint16_t *bblk, const uint16_t *qblk,
                                               const ListEntry *lists, int max_lists, const int *counts,
                                               const int *act, const int *rkeep, int lists_per_split, int col_tile,
                                               int target, int max_split, int exact_scan, uint32_t *winner,
                                               long long *winx, int *fb_list, int *fb_count, int *fb_done,
                                               const SpanBufs &sb)
{
    extern __shared__ int bk_all[];  // [warps][8][m+1]
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < g.R; r += gridDim.x * blockDim.x) {
        if (!rkeep[r]) {
            winner[r] = 0;
            winx[r] = unscreened_cross(g, ri[r], di);
        }
        fb_done[r] = 0;  // completion counters of the exact fallback
    }
    int *bk = bk_all + (threadIdx.x >> 5) * rescore_warp_ints(g.m);
    const int nkept = counts[0];
    for (int j = blockIdx.x * kRescoreWarps + (threadIdx.x >> 5); j < nkept; j += gridDim.x * kRescoreWarps)
        rescore_range<Wide>(g, ec, ri, di, bblk, qblk, lists, max_lists, counts, lists_per_split, col_tile, target,
                            max_split, exact_scan, winner, winx, fb_list, fb_count, act[j], bk, sb);
}

template <bool Wide>
__global__ void __launch_bounds__(32 * kRescoreWarps, 4)
    k_rescore(Geometry g, EpiConst ec, const RangeInfo *ri, const DomainInfo *di, const uint16_t *bblk,
              const uint16_t *qblk, const ListEntry *lists, int max_lists, const int *counts, const int *act,
              const int *rkeep, int lists_per_split, int col_tile, int target, int max_split, int exact_scan,
              uint32_t *winner, long long *winx, int *fb_list, int *fb_count, int *fb_done, SpanBufs sb)
{
    grid_dep_sync();
    rescore_blocks<Wide>(g, ec, ri, di, bblk, qblk, lists, max_lists, counts, act, rkeep, lists_per_split, col_tile,
                         target, max_split, exact_scan, winner, winx, fb_list, fb_count, fb_done, sb);
}

// Batched: one grid of persistent blocks over the ranges of all slices (in
// context order, ctx[s].r_begin the first); warp w takes every nw-th range,
// so the work of every slice is spread over all warps at once.
template <bool Wide>
__global__ void __launch_bounds__(32 * kRescoreWarps, 4)
    k_rescore_batch(const SliceCtx *__restrict__ ctx, int n, int total, int lists_per_split, int col_tile,
                    int exact_scan)
{
    extern __shared__ int bk_all[];  // [warps][8][m+1]
    grid_dep_sync();
    // ranges that are not screened: candidate 0 wins; exact-scan completion counters
    {
        const int nth = gridDim.x * blockDim.x;
        int s = 0;
        for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < total; gi += nth) {
            while (s + 1 < n && gi >= ctx[s + 1].r_begin) ++s;
            const EncBufs &b = ctx[s].b;
            const int r = gi - ctx[s].r_begin;
            if (!b.cb.rkeep[r]) {
                b.winner[r] = 0;
                b.winx[r] = unscreened_cross(ctx[s].g, b.ri[r], b.di);
            }
            fallback_done(ctx[s].g, b.partial)[r] = 0;
        }
    }
    const int nw = gridDim.x * kRescoreWarps;
    int s = 0;
    for (int gi = blockIdx.x * kRescoreWarps + (threadIdx.x >> 5); gi < total; gi += nw) {
        while (s + 1 < n && gi >= ctx[s + 1].r_begin) ++s;
        const SliceCtx &c = ctx[s];
        if (c.g.wide != Wide) continue;
        const int j = gi - c.r_begin;
        const EncBufs &b = c.b;
        if (j >= b.cb.counts[0]) continue;  // the screened ranges are the first counts[0]
        int *bk = bk_all + (threadIdx.x >> 5) * rescore_warp_ints(c.g.m);
        rescore_range<Wide>(c.g, c.ec, b.ri, b.di, b.bblk, b.qblk, b.lists, c.n_lists, b.cb.counts, lists_per_split,
                            col_tile, c.target, c.n_split, exact_scan, b.winner, b.winx, b.fb_list, b.fb_count,
                            b.cb.act[j], bk, span_bufs(c.g, c.n_lists, b.span, b.fb_count + 2));
    }
}



// The map of range r from its winner word wj (candidate index, bit 31: the
// winner came from an exact scan) and the exact statistics of the pair: codes
// decided as fp64_codes decides them (the FP32 shortcut where it provably
// agrees), the eq 8 residual exact in integers (64-bit unless the geometry
// needs 128, as in the re-score) and rounded once to FP64.
template <bool Wide>
__device__ __forceinline__ void write_map(const Geometry &g, const Stats &st, int r, uint32_t wj, const int *err,
                                          fic_map *maps)
{
    uint32_t ij = wj & 0x7fffffffu;
    if (ij >= (uint32_t)g.N) ij = 0;  // unreachable: every range has a winner
    int c, e;
    float sf, of;
    if (fast_codes(g, st, c, e)) {
        sf = s_hat_f(g, c);
        of = o_hat_f(g, e);
    } else {  // next to a rounding boundary: the FP64 sequence decides
        double sh, oh;
        fp64_codes(g, st, c, e, sh, oh);
        sf = (float)sh;
        of = (float)oh;
    }
    const double invD2 = 1.0 / ((double)(4 * g.Ls * g.Lo) * (double)(4 * g.Ls * g.Lo));
    fic_map mp;
    mp.range_idx = (uint32_t)r;
    mp.domain_idx = ij >> 3;
    mp.iso = ij & 7;
    mp.s_code = c;
    mp.o_code = e;
    mp.s = sf;
    mp.o = of;
    mp.info = ((wj & 0x80000000u) ? FIC_MAP_FALLBACK : 0u) | (*err ? FIC_MAP_ERROR : 0u);
    mp.err = (Wide ? u128_to_double((unsigned __int128)exact_err<true>(g, st, c, e))
                   : (double)(unsigned long long)exact_err<false>(g, st, c, e)) * invD2;
    maps[r] = mp;
}

// The map of one range whose winner an exact scan has just decided, by the
// calling warp (exact cross term over the lanes, the rest on lane 0).
template <bool Wide>
__device__ void finalize_range_warp(const Geometry &g, const RangeInfo *ri, const DomainInfo *di,
                                    const uint16_t *bblk, const uint16_t *qblk, int r, uint32_t wj, const int *err,
                                    fic_map *maps)
{
    const int lane = threadIdx.x & 31;
    uint32_t idx = wj & 0x7fffffffu;
    if (idx >= (uint32_t)g.N) idx = 0;
    const int d = idx >> 3;
    const SymFlags sf = sym_flags(idx & 7, g.n);
    long long X = 0;
    for (int i = lane; i < g.m; i += 32)
        X += (long long)qblk[(size_t)d * g.m + sym_src_index(sf, g.ln, i >> g.ln, i & (g.n - 1))] *
             bblk[(size_t)r * g.m + i];
    for (int off = 16; off > 0; off >>= 1) X += __shfl_xor_sync(0xffffffffu, X, off);
    if (lane == 0) {
        const RangeInfo rin = ri[r];
        const DomainInfo dd = di[d];
        write_map<Wide>(g, Stats{dd.Sq, dd.Sqq, rin.Sb, rin.Sbb, X}, r, wj, err, maps);
    }
}

// The range's pixels permuted for each symmetry, staged by the threads
// first, first + step, ...: bk[k*(m+1) + j] is the range pixel that S_k places
// over contracted-domain pixel j (the layout of stage_sym_pixels).
__device__ __forceinline__ void stage_sym_rows(const Geometry &g, const uint16_t *bblk, int r, int *bk, int first,
                                               int step)
{
    for (int i = first; i < g.m; i += step) {
        const int b = bblk[(size_t)r * g.m + i];
        const int y = i >> g.ln, x = i & (g.n - 1);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            int sy, sx;
            sym_src(k, g.n, y, x, sy, sx);
            bk[k * (g.m + 1) + (sy << g.ln) + sx] = b;
        }
    }
}

// Exhaustive exact scan of the ranges that failed certification, as work
// items (slot, chunk) over a grid of persistent blocks: an item scans one
// contiguous chunk of the candidates of range fb_list[slot] with exact integer
// decisions and writes its best (residual, index); the last item of a slot to
// finish (counted in done[slot], zeroed by the re-score) reduces the chunks
// and writes the winner, flagged as resolved by the fallback.
template <bool Wide>
__device__ __forceinline__ void full_scans(const Geometry &g, const RangeInfo *ri, const DomainInfo *di,
                                           const uint16_t *bblk, const uint16_t *qblk, const int *fb_list,
                                           const int *fb_count, int nch, Partial *part, int *done, uint32_t *winner,
                                           int first, int stride, const int *err, fic_map *maps)
{
    __shared__ int bk_s[8 * (kMaxM + 1)];
    __shared__ Partial w_s[8];
    __shared__ int last_s;
    __shared__ uint32_t fin_w;
    const int count = *fb_count;
    for (int item = first; item < count * nch; item += stride) {
        const int slot = item / nch, ch = item - slot * nch;
        const int lo = (int)((long long)g.N * ch / nch);
        const int hi = (int)((long long)g.N * (ch + 1) / nch);
        const int r = fb_list[slot];
        __syncthreads();  // bk_s and w_s of the previous item are no longer read
        stage_sym_rows(g, bblk, r, bk_s, threadIdx.x, blockDim.x);
        __syncthreads();
        const RangeInfo rin = ri[r];
        Stats st;
        st.Sb = rin.Sb;
        st.Sbb = rin.Sbb;
        typedef typename Exact<Wide>::U U;
        U best_e = ~(U)0;
        uint32_t best_i = 0xffffffffu;
        for (int idx = lo + threadIdx.x; idx < hi; idx += blockDim.x) {
            const int d = idx >> 3;
            const long long X = lane_cross(g, qblk, (uint32_t)idx, bk_s);
            const U er = exact_rational<Wide>(g, st, di[d], (long long)X);
            if (better(er, (uint32_t)idx, best_e, best_i)) {
                best_e = er;
                best_i = (uint32_t)idx;
            }
        }
        warp_argmin(best_e, best_i);
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0)
            w_s[w] = Partial{(unsigned long long)best_e, hi64(best_e), best_i, 0};
        __syncthreads();
        if (threadIdx.x == 0) {
            Partial b = w_s[0];
            for (int j = 1; j < (int)(blockDim.x >> 5); ++j) {
                const unsigned __int128 ej = ((unsigned __int128)w_s[j].hi << 64) | w_s[j].lo;
                const unsigned __int128 eb = ((unsigned __int128)b.hi << 64) | b.lo;
                if (better(ej, w_s[j].idx, eb, b.idx)) b = w_s[j];
            }
            part[(size_t)slot * nch + ch] = b;
            __threadfence();  // the partial is visible before the count says so
            last_s = atomicAdd(done + slot, 1) == nch - 1;
            if (last_s) {
                __threadfence();
                Partial bb{};
                bb.lo = __ldcg(&part[(size_t)slot * nch].lo);
                bb.hi = __ldcg(&part[(size_t)slot * nch].hi);
                bb.idx = __ldcg(&part[(size_t)slot * nch].idx);
                for (int j = 1; j < nch; ++j) {
                    const Partial *pj = part + (size_t)slot * nch + j;
                    const unsigned long long jl = __ldcg(&pj->lo), jh = __ldcg(&pj->hi);
                    const uint32_t ji = __ldcg(&pj->idx);
                    const unsigned __int128 ej = ((unsigned __int128)jh << 64) | jl;
                    const unsigned __int128 eb = ((unsigned __int128)bb.hi << 64) | bb.lo;
                    if (better(ej, ji, eb, bb.idx)) {
                        bb.lo = jl;
                        bb.hi = jh;
                        bb.idx = ji;
                    }
                }
                winner[r] = bb.idx | 0x80000000u;  // high bit: resolved by the fallback
                fin_w = bb.idx | 0x80000000u;
            }
        }
        if (maps) {  // the map of a range whose last chunk this was
            __syncthreads();
            if (last_s && threadIdx.x < 32) finalize_range_warp<Wide>(g, ri, di, bblk, qblk, r, fin_w, err, maps);
        }
    }
}

// Whether a re-scanned candidate (domain statistics dd and screening
// constants c4, exact cross term X) can be left out: with its code decided
// away from a rounding boundary, its FP32 screening key less the key's
// allowance lies above kcert, the certification's bound for the finalists'
// best residual, so its own residual exceeds that best and it can neither
// beat nor tie the winner (the test the certification applies to a list's
// last key).  Candidates next to a rounding boundary are always scored.
__device__ __forceinline__ bool scan_skip(const Geometry &g, const EpiConst &ec, const RangeEpi &re, long long Sb,
                                          const DomainInfo &dd, const float4 &c4, long long X, float kcert)
{
    const long long num = (long long)g.m * X - dd.Sq * Sb;  // exact
    const float Xt = __ll2float_rn(num) * ec.invm;
    float rho;
    const float c = epi_code(Xt, c4.x, 0.5f, ec, rho);
    if (fabsf(rho) > re.rho_lim) return false;
    const float key = epi_key(Xt, -0.0f, c, re.zb, c4, ec);
    return __fsub_rd(key, beta_key(re, key, ec)) > kcert;
}

// kcert of range r from the finalists' best exact residual the re-score left
// in sb.cert (rounded outward as in the certification).
template <bool Wide>
__device__ __forceinline__ float scan_kcert(const EpiConst &ec, const RangeInfo &rin, const Partial &cp)
{
    typedef typename Exact<Wide>::U U;
    const U e = Wide ? (U)(((unsigned __int128)cp.hi << 64) | cp.lo) : (U)cp.lo;
    return __fmul_ru(__fsub_ru(__fmul_ru(to_float_ru(e), ec.invD2_up), rin.sbbc), ec.two_ls);
}

// Exact scan of the candidates of one failed list (work item (range, list),
// one block each, for short queues; list_scans_warp below for long ones):
// list l = split * parts + part of a range holds the columns tile * col_tile
// + part * seg + [0, seg) of the tiles of its split, exactly as the search
// assigned them (compacted columns; dmap gives the domain).  Each item writes
// its best (residual, index); the last item of a range combines them with
// the finalists' best and writes the winner, flagged as resolved by an exact
// scan.
template <bool Wide>
__device__ __forceinline__ void list_scans_block(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                                           const DomainInfo *di, const float4 *dconst,
                                           const uint16_t *bblk, const uint16_t *qblk, const int *counts,
                                           const int *dmap, int col_tile, int target, int max_split,
                                           int lists_per_split, int max_lists, const SpanBufs &sb, uint32_t *winner,
                                           int first, int stride, const int *err, fic_map *maps)
{
    typedef typename Exact<Wide>::U U;
    __shared__ int bk_s[8 * (kMaxM + 1)];
    __shared__ Partial w_s[8];
    __shared__ int fin_s;
    __shared__ uint32_t fin_w;
    const int count = *sb.count;
    const int ncol = 8 * counts[2];
    const int tiles = (ncol + col_tile - 1) / col_tile;
    const int n_split = active_splits((counts[0] + 127) / 128, tiles, target, max_split, col_tile, g.m);
    const int n_lists = n_split * lists_per_split;
    const int seg = col_tile / lists_per_split;
    for (int item = first; item < count; item += stride) {
        const int code = sb.items[item];
        const int r = code >> 7, l = code & 127;
        const int sp = l / lists_per_split, part = l - sp * lists_per_split;
        const int t0 = split_tile(tiles, sp, n_split, col_tile), t1 = split_tile(tiles, sp + 1, n_split, col_tile);
        __syncthreads();  // bk_s and w_s of the previous item are no longer read
        stage_sym_rows(g, bblk, r, bk_s, threadIdx.x, blockDim.x);
        __syncthreads();
        const RangeInfo rin = ri[r];
        Stats st;
        st.Sb = rin.Sb;
        st.Sbb = rin.Sbb;
        const RangeEpi re = range_epi(rin, ec);
        const float kcert = scan_kcert<Wide>(ec, rin, sb.cert[r]);
        U best_e = ~(U)0;
        uint32_t best_i = 0xffffffffu;
        for (int i = threadIdx.x; i < (t1 - t0) * seg; i += blockDim.x) {
            const int ti = i / seg;
            const int c = (t0 + ti) * col_tile + part * seg + (i - ti * seg);
            if (c >= ncol) continue;
            const int d = dmap[c >> 3], k = c & 7;
            const uint32_t idx = (uint32_t)(d * 8 + k);
            const long long X = lane_cross(g, qblk, idx, bk_s);
            const DomainInfo dd = di[d];
            if (scan_skip(g, ec, re, st.Sb, dd, dconst[d], X, kcert)) continue;
            const U er = exact_rational<Wide>(g, st, dd, (long long)X);
            if (better(er, idx, best_e, best_i)) {
                best_e = er;
                best_i = idx;
            }
        }
        warp_argmin(best_e, best_i);
        if ((threadIdx.x & 31) == 0)
            w_s[threadIdx.x >> 5] = Partial{(unsigned long long)best_e, hi64(best_e), best_i, 0};
        __syncthreads();
        if (threadIdx.x == 0) {
            Partial b = w_s[0];
            for (int j = 1; j < (int)(blockDim.x >> 5); ++j) {
                const unsigned __int128 ej = ((unsigned __int128)w_s[j].hi << 64) | w_s[j].lo;
                const unsigned __int128 eb = ((unsigned __int128)b.hi << 64) | b.lo;
                if (better(ej, w_s[j].idx, eb, b.idx)) b = w_s[j];
            }
            Partial *sp_r = sb.part + (size_t)r * max_lists;
            sp_r[l] = b;
            __threadfence();  // the partial is visible before the count says so
            fin_s = 0;
            if (atomicSub(sb.pending + r, 1) == 1) {
                __threadfence();
                Partial bb = sb.cert[r];
                for (int j = 0; j < n_lists; ++j) {
                    const Partial *pj = sp_r + j;
                    const unsigned long long jl = __ldcg(&pj->lo), jh = __ldcg(&pj->hi);
                    const uint32_t ji = __ldcg(&pj->idx);
                    const unsigned __int128 ej = ((unsigned __int128)jh << 64) | jl;
                    const unsigned __int128 eb = ((unsigned __int128)bb.hi << 64) | bb.lo;
                    if (ji != 0xffffffffu && better(ej, ji, eb, bb.idx)) {
                        bb.lo = jl;
                        bb.hi = jh;
                        bb.idx = ji;
                    }
                }
                winner[r] = bb.idx | 0x80000000u;  // high bit: resolved by an exact scan
                fin_s = 1;
                fin_w = bb.idx | 0x80000000u;
            }
        }
        if (maps) {  // the map of a range whose last list this was
            __syncthreads();
            if (fin_s && threadIdx.x < 32) finalize_range_warp<Wide>(g, ri, di, bblk, qblk, r, fin_w, err, maps);
        }
    }
}

// The same scan with one warp per item, for long queues (more items than
// twice the blocks), where a warp rather than a block per item amortises the
// staging and the reduction.  bk: this warp's 8 (m+1) ints of shared memory;
// items first, first + stride, ...
template <bool Wide>
__device__ __forceinline__ void list_scans_warp(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                                           const DomainInfo *di, const float4 *dconst,
                                           const uint16_t *bblk, const uint16_t *qblk, const int *counts,
                                           const int *dmap, int col_tile, int target, int max_split,
                                           int lists_per_split, int max_lists, const SpanBufs &sb, uint32_t *winner,
                                           int *bk, int first, int stride, const int *err, fic_map *maps)
{
    typedef typename Exact<Wide>::U U;
    const int lane = threadIdx.x & 31;
    const int count = *sb.count;
    const int ncol = 8 * counts[2];
    const int tiles = (ncol + col_tile - 1) / col_tile;
    const int n_split = active_splits((counts[0] + 127) / 128, tiles, target, max_split, col_tile, g.m);
    const int n_lists = n_split * lists_per_split;
    const int seg = col_tile / lists_per_split;
    for (int item = first; item < count; item += stride) {
        const int code = sb.items[item];
        const int r = code >> 7, l = code & 127;
        const int sp = l / lists_per_split, part = l - sp * lists_per_split;
        const int t0 = split_tile(tiles, sp, n_split, col_tile), t1 = split_tile(tiles, sp + 1, n_split, col_tile);
        __syncwarp();  // bk of the previous item is no longer read
        stage_sym_rows(g, bblk, r, bk, lane, 32);
        __syncwarp();
        const RangeInfo rin = ri[r];
        Stats st;
        st.Sb = rin.Sb;
        st.Sbb = rin.Sbb;
        const RangeEpi re = range_epi(rin, ec);
        const float kcert = scan_kcert<Wide>(ec, rin, sb.cert[r]);
        U best_e = ~(U)0;
        uint32_t best_i = 0xffffffffu;
        for (int i = lane; i < (t1 - t0) * seg; i += 32) {
            const int ti = i / seg;
            const int c = (t0 + ti) * col_tile + part * seg + (i - ti * seg);
            if (c >= ncol) continue;
            const int d = dmap[c >> 3], k = c & 7;
            const uint32_t idx = (uint32_t)(d * 8 + k);
            const long long X = lane_cross(g, qblk, idx, bk);
            const DomainInfo dd = di[d];
            if (scan_skip(g, ec, re, st.Sb, dd, dconst[d], X, kcert)) continue;
            const U er = exact_rational<Wide>(g, st, dd, (long long)X);
            if (better(er, idx, best_e, best_i)) {
                best_e = er;
                best_i = idx;
            }
        }
        warp_argmin(best_e, best_i);
        uint32_t fin_w = 0;  // lane 0: the winner when this was the range's last list
        if (lane == 0) {
            Partial *sp_r = sb.part + (size_t)r * max_lists;
            sp_r[l] = Partial{(unsigned long long)best_e, hi64(best_e), best_i, 0};
            __threadfence();  // the partial is visible before the count says so
            if (atomicSub(sb.pending + r, 1) == 1) {
                __threadfence();
                Partial bb = sb.cert[r];
                for (int j = 0; j < n_lists; ++j) {
                    const Partial *pj = sp_r + j;
                    const unsigned long long jl = __ldcg(&pj->lo), jh = __ldcg(&pj->hi);
                    const uint32_t ji = __ldcg(&pj->idx);
                    const unsigned __int128 ej = ((unsigned __int128)jh << 64) | jl;
                    const unsigned __int128 eb = ((unsigned __int128)bb.hi << 64) | bb.lo;
                    if (ji != 0xffffffffu && better(ej, ji, eb, bb.idx)) {
                        bb.lo = jl;
                        bb.hi = jh;
                        bb.idx = ji;
                    }
                }
                winner[r] = bb.idx | 0x80000000u;  // high bit: resolved by an exact scan
                fin_w = bb.idx | 0x80000000u;
            }
        }
        fin_w = __shfl_sync(0xffffffffu, fin_w, 0);
        if (maps && fin_w != 0) finalize_range_warp<Wide>(g, ri, di, bblk, qblk, r, fin_w, err, maps);
    }
}

// FP64 codes of the winner (eq 9-12 in FP64, the operation order of the
// least-squares formulas) and its eq 8 residual, one thread of warp 0 per
// range so that every FP64 instruction works on 32 ranges.  The residual is
// evaluated exactly in integers and rounded once to FP64.  The block stages
// its 32 ranges' pixels and winners' 2x2 sums in shared memory with 16-byte
// loads (row pitch m+2 halves: an odd number of words, so lanes walking their
// own rows hit different banks), and its four warps each sum a quarter of the
// pixel rows of the exact cross term.
constexpr int kFinRanges = 32;
constexpr int kFinWarps = 4;
//
// When the re-score left every settled winner's cross term (winx) for the
// group, the maps need only the statistics (no staging): the usual case.
// scans_write: the exact scans write the maps of the ranges they resolve
// (winner bit 31), so this block leaves those out; otherwise (the batch,
// whose scans ran before) their cross terms are computed here.
template <bool Wide>
__device__ __forceinline__ void finalize_block(const Geometry &g, const RangeInfo *ri, const DomainInfo *di,
                                               const uint16_t *bblk, const uint16_t *qblk, const uint32_t *winner,
                                               const long long *winx, bool scans_write, const int *err,
                                               fic_map *maps, int bx)
{
    __shared__ uint32_t b_s[kFinRanges][(kMaxM + 2) / 2];
    __shared__ uint32_t q_s[kFinRanges][(kMaxM + 2) / 2];
    __shared__ uint32_t w_s[kFinRanges];
    __shared__ long long xw_s[kFinRanges];
    __shared__ int known_s;
    __shared__ long long x_s[kFinWarps][kFinRanges];
    __shared__ long long st_s[4][kFinRanges];  // Sq, Sqq of the winner's domain; Sb, Sbb of the range
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = bx * kFinRanges;
    const int nr = min(kFinRanges, g.R - r0);
    const int r = r0 + lane;
    const bool live = lane < nr;
    if (warp == 0) {
        const uint32_t w0 = live ? winner[r] : 0u;
        const long long x0 = live ? winx[r] : 0;
        w_s[lane] = w0;
        xw_s[lane] = x0;
        // no cross term needed here: no range, a winner the scans will decide
        // (and write), one they resolved when they write it; else it must be known
        const bool known = !live || win_pending(w0) || ((w0 & 0x80000000u) ? scans_write : x0 != kNoCross);
        const unsigned all = __ballot_sync(0xffffffffu, known);
        if (lane == 0) known_s = all == 0xffffffffu;
    }
    __syncthreads();
    if (known_s) {  // block-uniform
        constexpr int kPer = kFinRanges / kFinWarps;
        const int jr = warp * kPer + lane;
        if (lane >= kPer || jr >= nr) return;
        const uint32_t wj = w_s[jr];
        if (win_pending(wj) || (wj & 0x80000000u)) return;  // the scans write it
        uint32_t ij = wj;
        if (ij >= (uint32_t)g.N) ij = 0;  // unreachable: every range has a winner
        const RangeInfo rin = ri[r0 + jr];
        const DomainInfo dd = di[ij >> 3];
        write_map<Wide>(g, Stats{dd.Sq, dd.Sqq, rin.Sb, rin.Sbb, xw_s[jr]}, r0 + jr, wj, err, maps);
        return;
    }
    const uint32_t wv = w_s[lane];
    uint32_t idx = wv & 0x7fffffffu;
    if (idx >= (uint32_t)g.N) idx = 0;  // unreachable: every range has a winner
    const int d = idx >> 3, k = idx & 7;
    RangeInfo rin{};
    DomainInfo dd{};
    if (warp == 0 && live) {  // issued before the staging so that they overlap it
        rin = ri[r];
        dd = di[d];
    }
    const int pw = (g.m + 2) >> 1;  // row pitch in words
    const int lnv = 2 * g.ln - 3;   // log2 of the 16-byte vectors per row (m >= 16)
#pragma unroll 4
    for (int e = threadIdx.x; e < (nr << lnv); e += 32 * kFinWarps) {
        const int j = e >> lnv, v = e & ((1 << lnv) - 1);
        uint32_t jd = w_s[j] & 0x7fffffffu;
        if (jd >= (uint32_t)g.N) jd = 0;
        const uint4 bw = __ldg(reinterpret_cast<const uint4 *>(bblk + (size_t)(r0 + j) * g.m) + v);
        const uint4 qw = __ldg(reinterpret_cast<const uint4 *>(qblk + (size_t)(jd >> 3) * g.m) + v);
        uint32_t *bd = &b_s[0][0] + j * pw + 4 * v;
        uint32_t *qd = &q_s[0][0] + j * pw + 4 * v;
        bd[0] = bw.x, bd[1] = bw.y, bd[2] = bw.z, bd[3] = bw.w;
        qd[0] = qw.x, qd[1] = qw.y, qd[2] = qw.z, qd[3] = qw.w;
    }
    if (warp == 0 && live) {
        st_s[0][lane] = dd.Sq;
        st_s[1][lane] = dd.Sqq;
        st_s[2][lane] = rin.Sb;
        st_s[3][lane] = rin.Sbb;
    }
    __syncthreads();
    {
        // rows [warp*n/4, (warp+1)*n/4) of range `lane` (n >= 4)
        const uint16_t *brow = reinterpret_cast<const uint16_t *>(&b_s[0][0] + lane * pw);
        const uint16_t *qrow = reinterpret_cast<const uint16_t *>(&q_s[0][0] + lane * pw);
        const SymFlags sf = sym_flags(k, g.n);
        const int rows = g.n >> 2;
        long long X = 0;
        for (int y = warp * rows; y < (warp + 1) * rows; ++y) {
            uint32_t acc = 0;  // one row: n products of at most 4P * P, n <= 16
            for (int x = 0; x < g.n; ++x) acc += (uint32_t)qrow[sym_src_index(sf, g.ln, y, x)] * brow[(y << g.ln) + x];
            X += acc;
        }
        x_s[warp][lane] = X;
    }
    __syncthreads();
    // The FP64 part, a long dependent chain at the FP64 rate of this part:
    // spread over all warps of the block, kFinRanges / kFinWarps lanes each.
    constexpr int kPer = kFinRanges / kFinWarps;
    const int jr = warp * kPer + lane;  // the range of this lane
    if (lane >= kPer || jr >= nr) return;
    long long X = 0;
#pragma unroll
    for (int w = 0; w < kFinWarps; ++w) X += x_s[w][jr];
    const uint32_t wj = w_s[jr];
    if (win_pending(wj)) return;  // an exact scan decides it (and writes the map)
    write_map<Wide>(g, Stats{st_s[0][jr], st_s[1][jr], st_s[2][jr], st_s[3][jr], X}, r0 + jr, wj, err, maps);
}

// Shared memory of the list scans: 8 (m+1) ints per warp.
__host__ __device__ __forceinline__ size_t list_scan_smem(int m, int warps)
{
    return sizeof(int) * 8 * (size_t)warps * (size_t)(m + 1);
}

// The exact scans and the map output in one launch (persistent blocks of
// kFinWarps warps).  Each block first writes the maps of its groups of 32
// ranges whose winner the re-score settled, then takes exact-scan work items
// (usually there are none); the item that completes a range's scans writes
// its map.  A range's map is thus written once its winner is final, by
// whichever side sees it final (both write the same map).
template <bool Wide>
__global__ void __launch_bounds__(32 * kFinWarps) k_scans_finalize(Geometry g, const RangeInfo *ri,
                                                                   const DomainInfo *di, const uint16_t *bblk,
                                                                   const uint16_t *qblk, const int *fb_list,
                                                                   const int *fb_count, int nch, Partial *part,
                                                                   int *done, const int *counts, const int *dmap,
                                                                   int col_tile, int target, int max_split,
                                                                   int lists_per_split, int max_lists, SpanBufs sb,
                                                                   uint32_t *winner, const long long *winx,
                                                                   const int *err, fic_map *maps, EpiConst ec,
                                                                   const float4 *dconst)
{
    extern __shared__ int scan_sm[];  // [warps][8 (m+1)]
    grid_dep_sync();
    const int groups = (g.R + kFinRanges - 1) / kFinRanges;
    for (int gb = blockIdx.x; gb < groups; gb += gridDim.x) {
        finalize_block<Wide>(g, ri, di, bblk, qblk, winner, winx, true, err, maps, gb);
        __syncthreads();  // the block's staging is reused by its next group
    }
    full_scans<Wide>(g, ri, di, bblk, qblk, fb_list, fb_count, nch, part, done, winner, blockIdx.x, gridDim.x, err,
                     maps);
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (*sb.count > 2 * (int)gridDim.x)  // grid-uniform
        list_scans_warp<Wide>(g, ec, ri, di, dconst, bblk, qblk, counts, dmap, col_tile, target, max_split, lists_per_split,
                              max_lists, sb, winner, scan_sm + warp * 8 * (g.m + 1), blockIdx.x * nw + warp,
                              gridDim.x * nw, err, maps);
    else
        list_scans_block<Wide>(g, ec, ri, di, dconst, bblk, qblk, counts, dmap, col_tile, target, max_split, lists_per_split,
                               max_lists, sb, winner, blockIdx.x, gridDim.x, err, maps);
}

// Batched: the work items of all slices' queues form one sequence (the
// queue lengths of every slice are read at once, then prefix-summed), spread
// over the persistent blocks like a single queue.
template <bool Wide>
__global__ void __launch_bounds__(256) k_exact_scans_batch(const SliceCtx *__restrict__ ctx, int n,
                                                           int lists_per_split, int col_tile)
{
    __shared__ int fi_s[kMaxBatch + 1], li_s[kMaxBatch + 1];  // item prefixes: full scans, list scans
    extern __shared__ int scan_sm[];                          // [warps][8 (m+1)]
    grid_dep_sync();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const SliceCtx &c = ctx[i];
        const bool mine = c.g.wide == Wide;
        fi_s[i + 1] = mine ? c.b.fb_count[0] * fallback_chunks(c.g) : 0;
        li_s[i + 1] = mine ? c.b.fb_count[2] : 0;
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // inclusive scans, 32 slices at a time
        const int lane = threadIdx.x;
        int cf = 0, cl = 0;
        for (int i0 = 0; i0 < n; i0 += 32) {
            const int i = i0 + lane;
            int vf = i < n ? fi_s[i + 1] : 0, vl = i < n ? li_s[i + 1] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int yf = __shfl_up_sync(0xffffffffu, vf, o), yl = __shfl_up_sync(0xffffffffu, vl, o);
                if (lane >= o) {
                    vf += yf;
                    vl += yl;
                }
            }
            if (i < n) {
                fi_s[i + 1] = cf + vf;
                li_s[i + 1] = cl + vl;
            }
            cf += __shfl_sync(0xffffffffu, vf, 31);
            cl += __shfl_sync(0xffffffffu, vl, 31);
        }
        if (lane == 0) fi_s[0] = li_s[0] = 0;
    }
    __syncthreads();
    // full scans: block items b, b + G, ... of the global sequence
    const int b = blockIdx.x, G = gridDim.x;
    for (int s = 0; s < n; ++s) {
        const int nf = fi_s[s + 1] - fi_s[s];
        const int ff = ((b - fi_s[s]) % G + G) % G;  // this block's first item of the slice
        if (ff >= nf) continue;                      // block-uniform
        const SliceCtx &c = ctx[s];
        const EncBufs &e = c.b;
        full_scans<Wide>(c.g, e.ri, e.di, e.bblk, e.qblk, e.fb_list, e.fb_count, fallback_chunks(c.g),
                         reinterpret_cast<Partial *>(e.partial), fallback_done(c.g, e.partial), e.winner, ff, G,
                         nullptr, nullptr);
    }
    // list scans: one warp per item (warp items w, w + W, ... of the global
    // sequence) when the queues are long, else one block per item
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool by_warp = li_s[n] > 2 * G;  // grid-uniform
    const int w = by_warp ? b * nw + warp : b, W = by_warp ? G * nw : G;
    for (int s = 0; s < n; ++s) {
        const int nl = li_s[s + 1] - li_s[s];
        const int fl = ((w - li_s[s]) % W + W) % W;  // this warp's (block's) first item of the slice
        if (fl >= nl) continue;                      // warp- (block-) uniform
        const SliceCtx &c = ctx[s];
        const EncBufs &e = c.b;
        const SpanBufs sb = span_bufs(c.g, c.n_lists, e.span, e.fb_count + 2);
        if (by_warp)
            list_scans_warp<Wide>(c.g, c.ec, e.ri, e.di, e.dconst, e.bblk, e.qblk, e.cb.counts, e.cb.dmap, col_tile, c.target,
                                  c.n_split, lists_per_split, c.n_lists, sb, e.winner, scan_sm + warp * 8 * (c.g.m + 1),
                                  fl, W, nullptr, nullptr);
        else
            list_scans_block<Wide>(c.g, c.ec, e.ri, e.di, e.dconst, e.bblk, e.qblk, e.cb.counts, e.cb.dmap, col_tile, c.target,
                                   c.n_split, lists_per_split, c.n_lists, sb, e.winner, fl, W, nullptr, nullptr);
    }
}

template <bool Wide>
__global__ void __launch_bounds__(32 * kFinWarps) k_finalize_batch(const SliceCtx *__restrict__ ctx)
{
    grid_dep_sync();
    const SliceCtx c = ctx[blockIdx.y];
    if ((int)blockIdx.x * kFinRanges >= c.g.R) return;
    const EncBufs &b = c.b;
    finalize_block<Wide>(c.g, b.ri, b.di, b.bblk, b.qblk, b.winner, b.winx, false, b.err, c.maps, blockIdx.x);
}


cudaError_t launch_rescore(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                           const DomainInfo *di, const uint16_t *bblk, const uint16_t *qblk,
                           const ListEntry *lists, int max_lists, const int *counts, const int *act,
                           const int *rkeep, int lists_per_split, int col_tile, int target, int max_split, int n_sm,
                           int exact_scan, uint32_t *winner, long long *winx, int *fb_list, int *fb_count,
                           void *partial, void *span, cudaStream_t st)
{
    const SpanBufs sb = span_bufs(g, max_lists, span, fb_count + 2);
    const size_t smem = sizeof(int) * kRescoreWarps * rescore_warp_ints(g.m);
    // at most as many blocks as are resident at once (4 per SM at this size)
    const int blocks = std::max(1, std::min((g.R + kRescoreWarps - 1) / kRescoreWarps, 4 * n_sm));
    if (max_lists * kListK > 32 * kRescoreEnt) return cudaErrorInvalidValue;
    return launch_dep(g.wide ? k_rescore<true> : k_rescore<false>, dim3(blocks), dim3(32 * kRescoreWarps), smem, st,
                      g, ec, ri, di, bblk, qblk, lists, max_lists, counts, act, rkeep, lists_per_split, col_tile,
                      target, max_split, exact_scan, winner, winx, fb_list, fb_count, fallback_done(g, partial), sb);
}


// Partial results [R][chunks], then one completion counter per slot.
size_t fallback_partial_bytes(const Geometry &g)
{
    return sizeof(Partial) * (size_t)g.R * fallback_chunks(g) + sizeof(int) * (size_t)g.R;
}


cudaError_t launch_scans_finalize(const Geometry &g, const RangeInfo *ri, const DomainInfo *di, const uint16_t *bblk,
                                  const uint16_t *qblk, const int *fb_list, int *fb_count, void *partial,
                                  const int *counts, const int *dmap, int col_tile, int target, int max_split,
                                  int lists_per_split, int max_lists, void *span, uint32_t *winner,
                                  const long long *winx, const int *err, fic_map *maps, const EpiConst &ec,
                                  const float4 *dconst, int n_sm, cudaStream_t st)
{
    const int nch = fallback_chunks(g);
    Partial *part = reinterpret_cast<Partial *>(partial);
    const SpanBufs sb = span_bufs(g, max_lists, span, fb_count + 2);
    const size_t smem = list_scan_smem(g.m, kFinWarps);
    auto kern = g.wide ? k_scans_finalize<true> : k_scans_finalize<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // resident at once (the scans' work items are taken by stride); at least
    // one block per group of 32 ranges
    const int blocks = std::max((g.R + kFinRanges - 1) / kFinRanges, 3 * n_sm);
    return launch_dep(kern, dim3(blocks), dim3(32 * kFinWarps), smem, st, g, ri, di, bblk, qblk, fb_list,
                      (const int *)fb_count, nch, part, fallback_done(g, partial), counts, dmap, col_tile, target,
                      max_split, lists_per_split, max_lists, sb, winner, winx, err, maps, ec, dconst);
}

// Batched re-score and exact scans of n slices (max_m: the pixels per range,
// common to all slices; total_ranges: the sum over the slices).
cudaError_t launch_rescore_batch(const SliceCtx *ctx, int n, int total_ranges, bool any_wide, bool any_narrow,
                                 int max_m, int lists_per_split, int col_tile, int exact_scan, int n_sm,
                                 cudaStream_t st)
{
    const size_t smem = sizeof(int) * kRescoreWarps * rescore_warp_ints(max_m);
    const int blocks = 4 * n_sm;  // resident at once (4 per SM at this size)
    cudaError_t e;
    if (any_narrow && (e = launch_dep(k_rescore_batch<false>, dim3(blocks), dim3(32 * kRescoreWarps), smem, st, ctx, n,
                                      total_ranges, lists_per_split, col_tile, exact_scan)) != cudaSuccess)
        return e;
    if (any_wide && (e = launch_dep(k_rescore_batch<true>, dim3(blocks), dim3(32 * kRescoreWarps), smem, st, ctx, n,
                                    total_ranges, lists_per_split, col_tile, exact_scan)) != cudaSuccess)
        return e;
    const size_t ssm = list_scan_smem(max_m, 8);
    if ((e = cudaFuncSetAttribute(k_exact_scans_batch<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)ssm)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_exact_scans_batch<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)ssm)) != cudaSuccess)
        return e;
    if (any_narrow && (e = launch_dep(k_exact_scans_batch<false>, dim3(2 * n_sm), dim3(256), ssm, st, ctx, n,
                                      lists_per_split, col_tile)) != cudaSuccess)
        return e;
    if (any_wide && (e = launch_dep(k_exact_scans_batch<true>, dim3(2 * n_sm), dim3(256), ssm, st, ctx, n,
                                    lists_per_split, col_tile)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

// wide: some slice's residuals need 128-bit integers (128-bit arithmetic is
// exact for the others too)
cudaError_t launch_finalize_batch(const SliceCtx *ctx, int n, int ranges, bool wide, cudaStream_t st)
{
    return launch_dep(wide ? k_finalize_batch<true> : k_finalize_batch<false>,
                      dim3((ranges + kFinRanges - 1) / kFinRanges, n), dim3(32 * kFinWarps), 0, st, ctx);
}

}  // namespace fic
