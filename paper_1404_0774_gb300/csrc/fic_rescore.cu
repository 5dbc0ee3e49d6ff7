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
    const double o = __ddiv_rn(__dsub_rn(Sb, __dmul_rn(s_hat, Sa)), md);
    const double P = (double)g.P, Lo = (double)g.Lo;
    const double oc = o < -P ? -P : (o > P ? P : o);
    e = (int)round(__ddiv_rn(__dmul_rn(oc, Lo), P));
    o_hat = __ddiv_rn(__dmul_rn((double)e, P), Lo);
}

// Exact residual times D^2 for codes (c, e).
__device__ __int128 exact_err(const Geometry &g, const Stats &st, int c, int e)
{
    const __int128 A = (__int128)c * g.Lo;
    const __int128 Bo = (__int128)4 * g.Ls * e * g.P;
    const __int128 Dd = (__int128)4 * g.Ls * g.Lo;
    return A * A * st.Sqq + (__int128)g.m * Bo * Bo + Dd * Dd * st.Sbb + 2 * A * Bo * st.Sq -
           2 * A * Dd * st.X - 2 * Bo * Dd * st.Sb;
}

__device__ __forceinline__ bool better(unsigned __int128 e1, uint32_t i1, unsigned __int128 e2,
                                       uint32_t i2)
{
    return e1 < e2 || (e1 == e2 && i1 < i2);
}

__device__ __forceinline__ unsigned long long shfl64(unsigned long long v, int src)
{
    return __shfl_sync(0xffffffffu, v, src);
}

// Warp argmin over (err, idx).
__device__ void warp_argmin(unsigned __int128 &err, uint32_t &idx)
{
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long lo = shfl64((unsigned long long)err, (threadIdx.x & 31) ^ off);
        const unsigned long long hi = shfl64((unsigned long long)(err >> 64), (threadIdx.x & 31) ^ off);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, idx, off);
        const unsigned __int128 oe = ((unsigned __int128)hi << 64) | lo;
        if (better(oe, oi, err, idx)) {
            err = oe;
            idx = oi;
        }
    }
}

}  // namespace

__device__ __forceinline__ double u128_to_double(unsigned __int128 v)
{
    return (double)(unsigned long long)(v >> 64) * 18446744073709551616.0 + (double)(unsigned long long)v;
}

// Exact residual (times D^2) of one candidate whose cross term is X.
__device__ unsigned __int128 exact_candidate(const Geometry &g, Stats st, const DomainInfo *di, uint32_t idx,
                                             long long X)
{
    const DomainInfo dd = di[idx >> 3];
    st.Sq = dd.Sq;
    st.Sqq = dd.Sqq;
    st.X = X;
    int c, e;
    double sh, oh;
    fp64_codes(g, st, c, e, sh, oh);
    return (unsigned __int128)exact_err(g, st, c, e);
}

// Exact X of candidate idx for a range whose pixels b[] are spread over the
// warp (lane l holds pixels l, l+32, ...); every lane gets the sum.
__device__ long long warp_cross(const Geometry &g, const uint16_t *qblk, uint32_t idx, const int (&b)[kMaxM / 32])
{
    const int d = idx >> 3, k = idx & 7;
    const int lane = threadIdx.x & 31;
    long long acc = 0;
#pragma unroll
    for (int j = 0; j < kMaxM / 32; ++j) {
        const int i = lane + 32 * j;
        if (i < g.m) {
            int sy, sx;
            sym_src(k, g.n, i >> g.ln, i & (g.n - 1), sy, sx);
            acc += (long long)qblk[(size_t)d * g.m + (sy << g.ln) + sx] * b[j];
        }
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    return acc;
}

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
__device__ unsigned __int128 exact_rational(const Geometry &g, Stats st, const DomainInfo &dd, long long X)
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
    return (unsigned __int128)exact_err(g, st, c, e);
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
__global__ void k_rescore(Geometry g, EpiConst ec, const RangeInfo *ri, const DomainInfo *di,
                          const uint16_t *bblk, const uint16_t *qblk, const ListEntry *lists,
                          int max_lists, const int *counts, int lists_per_split, int col_tile, int target,
                          int max_split, int dense, uint32_t *winner, int *fb_list, int *fb_count)
{
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= g.R) return;  // warp-uniform
    const RangeInfo rin = ri[r];
    if (rin.shadow && !dense) {
        // constant range: num = 0 for every candidate, so s = 0, one offset and
        // one residual for all; the first candidate wins (Algorithm 2)
        if (lane == 0) winner[r] = 0;
        return;
    }
    int b[kMaxM / 32];
#pragma unroll
    for (int j = 0; j < kMaxM / 32; ++j) {
        const int i = lane + 32 * j;
        b[j] = i < g.m ? (int)bblk[(size_t)r * g.m + i] : 0;
    }
    // lists actually written by the search (its split count follows the kept counts)
    const int n_lists = lists_per_split *
                        active_splits((counts[0] + 127) / 128, (8 * counts[2] + col_tile - 1) / col_tile, target, max_split);
    const ListEntry *L = lists + (size_t)r * max_lists * kListK;
    const int nent = n_lists * kListK;
    float kb = __int_as_float(0x7f800000);
    uint32_t ib = 0xffffffffu;
    for (int f = lane; f < nent; f += 32) {
        const ListEntry e = L[f];
        if (e.idx != 0xffffffffu && (e.key < kb || (e.key == kb && e.idx < ib))) {
            kb = e.key;
            ib = e.idx;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const float ok = __shfl_xor_sync(0xffffffffu, kb, off);
        const uint32_t oi = __shfl_xor_sync(0xffffffffu, ib, off);
        if (ok < kb || (ok == kb && oi < ib)) {
            kb = ok;
            ib = oi;
        }
    }
    if (ib == 0xffffffffu) {  // no candidate was listed: exact rescan
        if (lane == 0) {
            winner[r] = 0xffffffffu;
            fb_list[atomicAdd(fb_count, 1)] = r;
        }
        return;
    }
    Stats st;
    st.Sb = rin.Sb;
    st.Sbb = rin.Sbb;
    const double invD2 = 1.0 / ((double)(4 * g.Ls * g.Lo) * (double)(4 * g.Ls * g.Lo));
    const double inv2ls = 1.0 / (2.0 * g.Ls);
    unsigned __int128 ue;
    {
        const long long X = warp_cross(g, qblk, ib, b);
        ue = exact_rational(g, st, di[ib >> 3], X);  // integer work, same on every lane
    }
    const double U = u128_to_double(ue) * invD2;
    // screening error allowance (the epilogue's), converted to residual units;
    // evaluated at the largest key that can still matter
    const RangeEpi re = range_epi(rin, ec);
    const float kreach = (float)((U - (double)rin.sbbc) * 2.0 * g.Ls);
    const float beta_k = fmaxf(beta_key(re, kb, ec), beta_key(re, fmaxf(kb, kreach), ec));
    const double betaE = (double)beta_k * inv2ls;
    const double sbbc = (double)rin.sbbc;

    unsigned __int128 best_e = ~(unsigned __int128)0;
    uint32_t best_i = 0xffffffffu;
    for (int f0 = 0; f0 < nent; f0 += 32) {
        const int f = f0 + lane;
        const ListEntry ent = f < nent ? L[f] : ListEntry{__int_as_float(0x7f800000), 0xffffffffu};
        const bool fin = ent.idx != 0xffffffffu && sbbc + (double)ent.key * inv2ls - betaE <= U;
        unsigned mask = __ballot_sync(0xffffffffu, fin);
        long long myX = 0;
        while (mask) {
            const int src = __ffs(mask) - 1;
            mask &= mask - 1;
            const uint32_t idx = __shfl_sync(0xffffffffu, ent.idx, src);
            const long long X = warp_cross(g, qblk, idx, b);
            if (lane == src) myX = X;
        }
        if (fin) {  // lanes re-score their own finalists in parallel (integer work)
            const unsigned __int128 er = exact_rational(g, st, di[ent.idx >> 3], myX);
            if (better(er, ent.idx, best_e, best_i)) {
                best_e = er;
                best_i = ent.idx;
            }
        }
    }
    // Flat domains were not screened: all their candidates have s = 0 and the
    // same residual, so only the first of them, (first flat domain, k = 0), can
    // win; it is a finalist of every range.
    const int dflat = counts[3];
    if (dflat >= 0) {
        const uint32_t fi = (uint32_t)dflat * 8;
        const long long X = warp_cross(g, qblk, fi, b);
        const unsigned __int128 er = exact_rational(g, st, di[dflat], X);
        if (lane == 0 && better(er, fi, best_e, best_i)) {
            best_e = er;
            best_i = fi;
        }
    }
    warp_argmin(best_e, best_i);
    const double Estar = u128_to_double(best_e) * invD2;
    bool cert = true;
    for (int l = lane; l < n_lists; l += 32) {
        // a full list's unlisted candidates have residual >= its last key less
        // the allowance at that key; that bound must clear the winner strictly
        const ListEntry last = L[l * kListK + kListK - 1];
        if (last.idx == 0xffffffffu) continue;
        const double bl = (double)beta_key(re, last.key, ec) * inv2ls;
        if (!(sbbc + (double)last.key * inv2ls - bl > Estar * (1.0 + 1e-12) + 1e-12)) cert = false;
    }
    cert = __all_sync(0xffffffffu, cert);
    if (lane == 0) {
        winner[r] = best_i;
        if (!cert) fb_list[atomicAdd(fb_count, 1)] = r;
    }
}

struct Partial {
    unsigned long long lo, hi;
    uint32_t idx, pad;
};

// Exhaustive exact scan of the ranges that failed certification.  Each range
// is split over gridDim.x CTAs (blockIdx.x = candidate chunk); each CTA writes
// its best (residual, index) to part[slot][chunk].
__global__ void __launch_bounds__(256) k_fallback(Geometry g, const RangeInfo *ri, const DomainInfo *di,
                                                  const uint16_t *bblk, const uint16_t *qblk,
                                                  const int *fb_list, const int *fb_count, Partial *part)
{
    __shared__ int b_s[kMaxM];
    __shared__ Partial w_s[8];
    const int count = *fb_count;
    const int nch = gridDim.x;
    const int lo = (int)((long long)g.N * blockIdx.x / nch);
    const int hi = (int)((long long)g.N * (blockIdx.x + 1) / nch);
    for (int slot = blockIdx.y; slot < count; slot += gridDim.y) {
        const int r = fb_list[slot];
        __syncthreads();
        for (int i = threadIdx.x; i < g.m; i += blockDim.x) b_s[i] = bblk[(size_t)r * g.m + i];
        __syncthreads();
        const RangeInfo rin = ri[r];
        Stats st;
        st.Sb = rin.Sb;
        st.Sbb = rin.Sbb;
        unsigned __int128 best_e = ~(unsigned __int128)0;
        uint32_t best_i = 0xffffffffu;
        for (int idx = lo + threadIdx.x; idx < hi; idx += blockDim.x) {
            const int d = idx >> 3, k = idx & 7;
            unsigned long long X = 0;
            for (int i = 0; i < g.m; ++i) {
                int sy, sx;
                sym_src(k, g.n, i >> g.ln, i & (g.n - 1), sy, sx);
                X += (unsigned long long)((unsigned)qblk[(size_t)d * g.m + sy * g.n + sx] * (unsigned)b_s[i]);
            }
            const unsigned __int128 er = exact_rational(g, st, di[d], (long long)X);
            if (better(er, (uint32_t)idx, best_e, best_i)) {
                best_e = er;
                best_i = (uint32_t)idx;
            }
        }
        warp_argmin(best_e, best_i);
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) w_s[w] = Partial{(unsigned long long)best_e, (unsigned long long)(best_e >> 64), best_i, 0};
        __syncthreads();
        if (threadIdx.x == 0) {
            Partial b = w_s[0];
            for (int j = 1; j < (int)(blockDim.x >> 5); ++j) {
                const unsigned __int128 ej = ((unsigned __int128)w_s[j].hi << 64) | w_s[j].lo;
                const unsigned __int128 eb = ((unsigned __int128)b.hi << 64) | b.lo;
                if (better(ej, w_s[j].idx, eb, b.idx)) b = w_s[j];
            }
            part[(size_t)slot * nch + blockIdx.x] = b;
        }
    }
}

__global__ void k_fallback_reduce(int nch, const int *fb_list, const int *fb_count, const Partial *part,
                                  uint32_t *winner)
{
    const int count = *fb_count;
    for (int slot = blockIdx.x * blockDim.x + threadIdx.x; slot < count; slot += gridDim.x * blockDim.x) {
        Partial b = part[(size_t)slot * nch];
        for (int j = 1; j < nch; ++j) {
            const Partial pj = part[(size_t)slot * nch + j];
            const unsigned __int128 ej = ((unsigned __int128)pj.hi << 64) | pj.lo;
            const unsigned __int128 eb = ((unsigned __int128)b.hi << 64) | b.lo;
            if (better(ej, pj.idx, eb, b.idx)) b = pj;
        }
        winner[fb_list[slot]] = b.idx | 0x80000000u;  // high bit: resolved by the fallback
    }
}

// FP64 codes of the winner (eq 9-12 in FP64, the operation order of the
// least-squares formulas) and its eq 8 residual, one thread per range so that
// every FP64 instruction works on 32 ranges.  The residual is evaluated
// exactly in integers and rounded once to FP64.  The range's pixels and the
// winner's 2x2 sums are staged in shared memory by the whole block.
constexpr int kFinRanges = 32;
__global__ void __launch_bounds__(128) k_finalize(Geometry g, const RangeInfo *ri, const DomainInfo *di,
                                                  const uint16_t *bblk, const uint16_t *qblk,
                                                  const uint32_t *winner, const int *err, fic_map *maps)
{
    __shared__ uint16_t b_s[kFinRanges][kMaxM + 2];  // row pitch of 129 words: conflict-free
    __shared__ uint16_t q_s[kFinRanges][kMaxM + 2];
    __shared__ uint32_t w_s[kFinRanges];
    const int r0 = blockIdx.x * kFinRanges;
    const int nr = min(kFinRanges, g.R - r0);
    for (int j = threadIdx.x; j < nr; j += blockDim.x) w_s[j] = winner[r0 + j];
    __syncthreads();
    const int lm = 2 * g.ln;
    for (int e = threadIdx.x; e < nr * g.m; e += blockDim.x) {
        const int j = e >> lm, i = e & (g.m - 1);
        uint32_t idx = w_s[j] & 0x7fffffffu;
        if (idx >= (uint32_t)g.N) idx = 0;  // unreachable: every range has a winner
        b_s[j][i] = bblk[(size_t)(r0 + j) * g.m + i];
        q_s[j][i] = qblk[(size_t)(idx >> 3) * g.m + i];
    }
    __syncthreads();
    const int j = threadIdx.x;
    if (j >= nr) return;
    const int r = r0 + j;
    const uint32_t wv = w_s[j];
    uint32_t idx = wv & 0x7fffffffu;
    if (idx >= (uint32_t)g.N) idx = 0;
    const int d = idx >> 3, k = idx & 7;
    const RangeInfo rin = ri[r];
    const DomainInfo dd = di[d];
    long long X = 0;
    for (int i = 0; i < g.m; ++i) {
        int sy, sx;
        sym_src(k, g.n, i >> g.ln, i & (g.n - 1), sy, sx);
        X += (long long)q_s[j][(sy << g.ln) + sx] * b_s[j][i];
    }
    Stats st{dd.Sq, dd.Sqq, rin.Sb, rin.Sbb, X};
    int c, e;
    double sh, oh;
    fp64_codes(g, st, c, e, sh, oh);
    const double invD2 = 1.0 / ((double)(4 * g.Ls * g.Lo) * (double)(4 * g.Ls * g.Lo));
    fic_map mp;
    mp.range_idx = (uint32_t)r;
    mp.domain_idx = (uint32_t)d;
    mp.iso = k;
    mp.s_code = c;
    mp.o_code = e;
    mp.s = (float)sh;
    mp.o = (float)oh;
    mp.info = ((wv & 0x80000000u) ? FIC_MAP_FALLBACK : 0u) | (*err ? FIC_MAP_ERROR : 0u);
    mp.err = u128_to_double((unsigned __int128)exact_err(g, st, c, e)) * invD2;
    maps[r] = mp;
}

cudaError_t launch_rescore(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                           const DomainInfo *di, const uint16_t *bblk, const uint16_t *qblk,
                           const ListEntry *lists, int max_lists, const int *counts, int lists_per_split,
                           int col_tile, int target, int max_split, int dense, uint32_t *winner, int *fb_list,
                           int *fb_count, cudaStream_t st)
{
    k_rescore<<<(g.R + 3) / 4, 128, 0, st>>>(g, ec, ri, di, bblk, qblk, lists, max_lists, counts, lists_per_split,
                                             col_tile, target, max_split, dense, winner, fb_list, fb_count);
    return cudaGetLastError();
}

int fallback_chunks(const Geometry &g) { return std::min(64, std::max(1, g.N / 1024)); }

size_t fallback_partial_bytes(const Geometry &g)
{
    return sizeof(Partial) * (size_t)g.R * fallback_chunks(g);
}

cudaError_t launch_fallback(const Geometry &g, const RangeInfo *ri, const DomainInfo *di,
                            const uint16_t *bblk, const uint16_t *qblk, const int *fb_list,
                            const int *fb_count, void *partial, uint32_t *winner, cudaStream_t st)
{
    const int nch = fallback_chunks(g);
    Partial *part = reinterpret_cast<Partial *>(partial);
    k_fallback<<<dim3(nch, 16), 256, 0, st>>>(g, ri, di, bblk, qblk, fb_list, fb_count, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_fallback_reduce<<<4, 256, 0, st>>>(nch, fb_list, fb_count, part, winner);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Geometry &g, const RangeInfo *ri, const DomainInfo *di,
                            const uint16_t *bblk, const uint16_t *qblk, const uint32_t *winner,
                            const int *err, fic_map *maps, cudaStream_t st)
{
    k_finalize<<<(g.R + kFinRanges - 1) / kFinRanges, 128, 0, st>>>(g, ri, di, bblk, qblk, winner, err, maps);
    return cudaGetLastError();
}

}  // namespace fic
