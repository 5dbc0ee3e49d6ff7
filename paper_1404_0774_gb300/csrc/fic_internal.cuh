// Internal definitions shared by the CUDA translation units of libfic.
//
// Notation (Haque et al., arXiv 1404.0774, Section V): range block b (n x n,
// m = n*n pixels), domain block (2n x 2n) contracted by the 2x2 mean to
// a = q/4 where q is the 2x2 *sum* (an integer), symmetry S_k, least squares
// s, o (eq 9-12), residual R (eq 8).
//
// Integer statistics (all exact):
//   Sb = sum b, Sbb = sum b^2                      per range
//   Sq = sum q, Sqq = sum q^2                      per domain (symmetry-invariant)
//   X  = sum_i q_i b_i                              per (range, domain, symmetry)
//   num = m*X - Sq*Sb,  den = m*Sqq - Sq^2        so that s = 4*num/den
// The search kernels see centred operands q' = q - c_d, b' = b - c_r and
// compute Xt = sum q'b' - e_r*f_d/m = num/m, where c_d, c_r are integer
// centres, f_d = Sq - m*c_d and e_r = Sb - m*c_r.
//
// FP32 screening key of a candidate with s code c and o residual w:
//   key = c*(c*kappa - Xt) + lambda*w^2 = 2*Ls*(R - Sbb_c)
// with kappa = den/(8*m*Ls), Sbb_c = Sbb - Sb^2/m, and w = z - e*G the
// residue of z = 4*Ls*Sb - c*Sq against the o grid (G = 4*Ls*m*P/Lo, e the
// rounded o code), lambda = 2*Ls*m*(P/Lo)^2/G^2.  Ranking by key within a
// range is ranking by R.  Candidates are kept in small per-range top-K lists
// and every list entry is re-scored exactly afterwards.
#pragma once

#include <cuda_fp16.h>
#include <utility>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fic.h"

namespace fic {

// Programmatic dependent launch: a pipeline kernel may be scheduled while its
// predecessor in the stream drains.  Each one waits for the predecessor's
// completion (and memory) before touching global memory, then lets its own
// successor be scheduled.
__device__ __forceinline__ void grid_dep_sync()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

constexpr int kListK = 4;          // entries per candidate list
// A list entry's idx carries the candidate index (8d + k, < 2^31) and, in bit
// 31, whether its key is clean: code not next to a rounding boundary and
// offset not clamped, so that the key bounds the exact residual from above up
// to the screening allowance.  An empty entry is 0xffffffff.
constexpr uint32_t kCleanBit = 0x80000000u;
constexpr uint32_t kIdxMask = 0x7fffffffu;
constexpr int kMaxM = 256;         // largest range (16 x 16)
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: x + kMagic rounds x to an integer

struct Geometry {
    int w, h, pitch;   // image size and row pitch (elements)
    int n, t, m;       // range size, domain stride, pixels per range
    int ln;            // log2(n): n is a power of two
    int nx, ny, R;     // ranges per row / column / total
    int U, V, D;       // domains per row / column / total
    int N;             // candidates = 8*D
    int B, P;          // bit depth, 2^B - 1
    int s_bits, o_bits, Ls, Lo;
    int split_hilo;    // 1 when q' must be split into two exact FP16 parts
    int KP;            // FP16 operand row length (tensor-core layout)
    int mod_g;         // 1 when G is an integer (z may be reduced mod G)
    int Gi;            // G when mod_g (< 2^31), else 0
    int wide;          // exact residuals need 128-bit integers (else 64-bit suffice)
    double G;          // 4*Ls*m*P/Lo
};

struct RangeInfo {
    long long Sb, Sbb;  // exact sums
    int c_r, e_r;       // centre and e_r = Sb - m*c_r
    float sbbc;         // Sbb - Sb^2/m
    float zb;           // 4*Ls*Sb (reduced mod G when mod_g)
    float bp2;          // sum (b - c_r)^2
    float rho_lim;      // |rho| above this: the s code may differ from FP64's
    float beta_a;       // key rounding allowance (see beta_key)
    float beta_q;       // cross-term accumulation allowance factor (0: exact)
    int shadow;         // constant block: every candidate has s = 0 and one residual
    int pad;
};

struct DomainInfo {
    long long Sq, Sqq;  // exact sums of the 2x2 sums q
    int c_d, f_d;       // centre and f_d = Sq - m*c_d
    float qp2;          // sum (q - c_d)^2
    float pad;
};

// Per-domain column constants of the epilogue.
//   x: alpha = 2*m/den (0 for a flat domain) so that Ls*clamp(s) = 2*Ls*sat(Xt*alpha+1/2) - Ls
//   y: sqz   = Sq (reduced mod G when mod_g)
//   z: kappa = den/(8*m*Ls)
//   w: Sq as float (exact)
struct EpiConst {
    float two_ls, ls, inv2ls;
    float G, invG;
    float lambda;
    float delta_o;      // m*(P/(2*Lo))^2: largest offset-rounding term of the residual
    float beta_o;       // key error from an o code decided next to its rounding boundary
    float sqrtm4;       // sqrt(m)/4
    float inv4ls, invm, pmax;  // 1/(4*Ls), 1/m, P (offset clamp detection)
    float near_slack;   // kappa * near_slack bounds how far below c*y the key of the other code can fall
    float invD2_up;     // FP32 upper bound of 1/(4*Ls*Lo)^2 (exact residuals are integers / D^2)
    float qmax;         // upper bound of the offset term lambda*w^2 of any candidate's key (w the o-grid residue)
};

// Per-thread constants of the range the thread screens.
struct RangeEpi {
    float zb, rho_lim;
    float sbbc, sqrt_sbbc;
    float bA, bQ;       // error allowance terms, see beta_key
    float Sb;           // sum b (exact as float)
    int shadow;
};

struct ListEntry {
    float key;
    uint32_t idx;
};

// Per-thread state: one top-K list of one range.
struct ListState {
    float key[kListK];
    uint32_t idx[kListK];
    int has_zero;       // an s-code-0 candidate is (or was) in the list
    float T;            // best clean key seen for this range (own or shared)
    float tw;           // T + 3*beta(T): larger keys cannot reach the winner
    float Tpub;         // value last published to (or read from) the shared per-range best
};

__device__ __forceinline__ int f2ord(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}

__device__ __forceinline__ float ord2f(int o) { return __int_as_float(o >= 0 ? o : o ^ 0x7fffffff); }

// Allowance (key units, key = 2*Ls*(R - Sbb_c)) for |key - exact| of any
// candidate whose residual is within reach of key T:
//   FP32 rounding of the key terms, the cross-term accumulation error (zero
//   unless centred products can exceed 2^23, see bQ), and the o-code decision
//   next to its rounding boundary.
__device__ __forceinline__ float beta_key(const RangeEpi &re, float T, const EpiConst &ec)
{
    const float ET = fmaxf(0.0f, fmaf(T, ec.inv2ls, re.sbbc));
    return re.bA + ec.beta_o + 3.814697265625e-6f * (fabsf(T) + 2.0f * ec.two_ls * ET) +
           re.bQ * (re.sqrt_sbbc + sqrtf(ET + ec.delta_o) + ec.sqrtm4);
}

__device__ __forceinline__ void list_init(ListState &L)
{
#pragma unroll
    for (int i = 0; i < kListK; ++i) {
        L.key[i] = __int_as_float(0x7f800000);  // +inf
        L.idx[i] = 0xffffffffu;
    }
    L.has_zero = 0;
    L.T = __int_as_float(0x7f800000);
    L.tw = __int_as_float(0x7f800000);
    L.Tpub = __int_as_float(0x7f800000);
}

// Adopt a better shared best key.
__device__ __forceinline__ void list_adopt(ListState &L, float T, const RangeEpi &re, const EpiConst &ec)
{
    if (T < L.T) {
        L.T = T;
        L.tw = T + 3.0f * beta_key(re, T, ec);
    }
}

// Sorted insertion; equal keys keep the earlier (lower-index) entry first.
__device__ __forceinline__ void list_insert(ListState &L, float key, uint32_t idx)
{
    if (!(key < L.key[kListK - 1])) return;
    float k = key;
    uint32_t id = idx;
#pragma unroll
    for (int i = 0; i < kListK; ++i) {
        const bool take = k < L.key[i];
        const float tk = L.key[i];
        const uint32_t ti = L.idx[i];
        if (take) {
            L.key[i] = k;
            L.idx[i] = id;
            k = tk;
            id = ti;
        }
    }
}

// The centring correction of a cross term accumulated without it:
// Xt = X' + corr, corr = -e_r f_d / m, where f_d / m = Sq/m - round(Sq/m) is
// recovered exactly from Sq (m a power of two, Sq < 2^24).  With er = 0 (a
// cross term that already includes it) corr is 0.  Exact in FP32.
__device__ __forceinline__ float epi_corr(float er, float Sq, const EpiConst &ec)
{
    const float a = Sq * ec.invm;
    return -er * (a - floorf(a + 0.5f));
}

// Code decision of one candidate from X' (Xt = X' + corr): returns c
// (integer-valued float) and rho.  bq = 1/2 + corr * alpha.
__device__ __forceinline__ float epi_code(float X, float alpha, float bq, const EpiConst &ec, float &rho)
{
    const float u = __saturatef(fmaf(X, alpha, bq));
    const float r = fmaf(u, ec.two_ls, -ec.ls);  // Ls * clamp(s, -1, 1)
    const float c = __fsub_rn(__fadd_rn(r, kMagic), kMagic);
    rho = __fsub_rn(r, c);
    return c;
}

// Screening key for a fixed code c, from X' and mcorr = -corr.
__device__ __forceinline__ float epi_key(float X, float mcorr, float c, float zb, float4 dc, const EpiConst &ec)
{
    const float z = fmaf(c, -dc.y, zb);
    const float e = __fsub_rn(fmaf(z, ec.invG, kMagic), kMagic);
    const float wv = fmaf(e, -ec.G, z);
    const float y = fmaf(c, dc.z, __fsub_rn(mcorr, X));
    const float cy = __fmul_rn(c, y);
    return fmaf(__fmul_rn(wv, ec.lambda), wv, cy);
}

// Packed FP32 pairs (sm_100 family .f32x2 arithmetic, round to nearest):
// two candidates per instruction, each lane computing exactly what the scalar
// operation would.
typedef unsigned long long f32x2_t;

__device__ __forceinline__ f32x2_t pk2(float lo, float hi)
{
    f32x2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void upk2(f32x2_t v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f32x2_t fma2(f32x2_t a, f32x2_t b, f32x2_t c)
{
    f32x2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2_t add2(f32x2_t a, f32x2_t b)
{
    f32x2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2_t sub2(f32x2_t a, f32x2_t b)
{
    f32x2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2_t mul2(f32x2_t a, f32x2_t b)
{
    f32x2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Main pass over 32 consecutive candidates (4 domains x 8 symmetries) with
// cross terms X[] = X' (the cross term less the centring correction of
// epi_corr, er = e_r; er = 0 when X[] already is Xt; the correction is
// folded into the code's offset and the key's -X' term, so it costs nothing
// per candidate).  Branch-free, two candidates (same domain, so same column
// constants) per packed instruction; the keys are bit-identical to
// epi_code/epi_key.  Returns the mask of candidates whose key is below `thr`
// (bit j for X[j]): the ones a rare pass must visit.  A code decided next to its rounding
// boundary (|rho| > rho_lim) may be the neighbouring one in FP64; its key is
// then replaced by a lower bound of both codes' keys (see below), so that
// such a candidate costs a rare pass only when it could enter the list.
// Lanes beyond the ragged end carry X = NaN (their keys are NaN and compare
// false everywhere).  zpen: added to the key of s-code-0 candidates (their
// residual is one value per range; once the list holds one, the others need
// never be looked at).
//
// Lower bound for a near-boundary candidate.  With r = Xt/(2*kappa) (the
// unrounded Ls*s) the s part of the key is f(c) = c*(c*kappa - Xt) =
// kappa*((c - r)^2 - r^2), so for the neighbour c2 = c + sign(rho):
// f(c2) - f(c) = kappa*(1 - 2|rho|) >= -2*kappa*e, e the FP32 error of rho
// (at most 7*Ls*2^-24).  The FP32 evaluations of c*y and c2*y2 each carry at
// most 8*Ls^2*kappa*2^-24, and lambda*w^2 >= 0, so both keys are at least
// c*y - kappa*near_slack with near_slack = (32*Ls^2 + 16*Ls)*2^-24.
//
// kNearPass: every near-boundary candidate goes to the rare pass instead
// (the tensor-core search, whose near band is about 3e-4 wide), and the
// mask is assembled from sign bits: bit (k - thr < 0) | (rho^2 >= lim^2),
// with lim^2 rounded down so the band holds every |rho| > rho_lim.
template <bool kNearPass = false>
__device__ __forceinline__ uint32_t epi_keys32(const float (&X)[32], const float4 (&dc)[4], float zb, float rho_lim,
                                               float er, const EpiConst &ec, float thr, float zpen)
{
    uint32_t mask = 0, far = 0;  // kNearPass: bit-reversed masks of k < thr, of |rho| below the band
    const f32x2_t thr2 = pk2(thr, thr);
    const float mlim2 = -__fmul_rd(rho_lim, rho_lim);
    const f32x2_t mlim = pk2(mlim2, mlim2);
    const f32x2_t two_ls = pk2(ec.two_ls, ec.two_ls), mls = pk2(-ec.ls, -ec.ls);
    const f32x2_t mag = pk2(kMagic, kMagic), zb2 = pk2(zb, zb), invg = pk2(ec.invG, ec.invG);
    const f32x2_t mg = pk2(-ec.G, -ec.G), lam = pk2(ec.lambda, ec.lambda), zp = pk2(zpen, zpen);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 c4 = dc[q];
        const f32x2_t msqz = pk2(-c4.y, -c4.y), kap = pk2(c4.z, c4.z);
        const float sl = -c4.z * ec.near_slack;
        const f32x2_t msl = pk2(sl, sl);
        const float corr = epi_corr(er, c4.w, ec);
        const float bq = fmaf(corr, c4.x, 0.5f);
        const f32x2_t mcorr = pk2(-corr, -corr);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int j = q * 8 + 2 * h;
            const float u0 = __saturatef(fmaf(X[j], c4.x, bq));
            const float u1 = __saturatef(fmaf(X[j + 1], c4.x, bq));
            const f32x2_t x = pk2(X[j], X[j + 1]);
            const f32x2_t r = fma2(pk2(u0, u1), two_ls, mls);  // Ls * clamp(s, -1, 1)
            const f32x2_t c = sub2(add2(r, mag), mag);          // rounded code
            const f32x2_t rho = sub2(r, c);
            float c0, c1, p0, p1;
            upk2(c, c0, c1);
            upk2(rho, p0, p1);
            const float zero0 = __saturatef(fmaf(c0, -c0, 1.0f));  // 1 for c = 0, else 0
            const float zero1 = __saturatef(fmaf(c1, -c1, 1.0f));
            const f32x2_t z = fma2(c, msqz, zb2);
            const f32x2_t e = sub2(fma2(z, invg, mag), mag);
            const f32x2_t wv = fma2(e, mg, z);
            const f32x2_t y = fma2(c, kap, sub2(mcorr, x));
            const f32x2_t cy = mul2(c, y);
            f32x2_t k = fma2(mul2(wv, lam), wv, cy);
            k = fma2(pk2(zero0, zero1), zp, k);
            if (kNearPass) {
                float d0, d1, t0, t1;
                upk2(sub2(k, thr2), d0, d1);
                upk2(fma2(rho, rho, mlim), t0, t1);
                mask = __funnelshift_l(__float_as_uint(d0), mask, 1);  // (mask << 1) | sign bit
                mask = __funnelshift_l(__float_as_uint(d1), mask, 1);
                far = __funnelshift_l(__float_as_uint(t0), far, 1);
                far = __funnelshift_l(__float_as_uint(t1), far, 1);
            } else {
                const f32x2_t lo = add2(cy, msl);
                float k0, k1, l0, l1;
                upk2(k, k0, k1);
                upk2(lo, l0, l1);
                k0 = fabsf(p0) > rho_lim ? l0 : k0;
                k1 = fabsf(p1) > rho_lim ? l1 : k1;
                mask |= (k0 < thr ? 1u : 0u) << j;
                mask |= (k1 < thr ? 1u : 0u) << (j + 1);
            }
        }
    }
    return kNearPass ? __brev(mask | ~far) : mask;
}

__device__ __forceinline__ float4 pick4(const float4 (&dc)[4], int q)
{
    return q == 0 ? dc[0] : (q == 1 ? dc[1] : (q == 2 ? dc[2] : dc[3]));
}

// Rare pass for one thread: cross terms X' staged in shared memory at
// xrow[j*stride] (er as for epi_keys32); only the candidates of `mask` (the main pass's keys below
// its threshold, a superset of what can still enter the list) are visited,
// their keys recomputed (bit-identical to the main pass).  Handles codes next
// to a rounding boundary (the key becomes the smaller of the two neighbouring
// codes' keys: a lower bound of the residual FP64 decides) and list insertion
// with s-code-0 de-duplication (all such candidates of a range have one
// residual).  od[q]: original index of the chunk's q-th domain (the search
// may skip flat domains, so consecutive columns need not be consecutive
// domains).
static __device__ __forceinline__ void epi_rare(const float *xrow, int stride, const int (&od)[4],
                                                const float4 (&dc)[4], float er, const RangeEpi &re,
                                                const EpiConst &ec, ListState &L, uint32_t mask)
{
#pragma unroll 1
    while (mask) {
        const int j = __ffs(mask) - 1;
        mask &= mask - 1;
        const float x = xrow[j * stride];
        const float4 c4 = pick4(dc, j >> 3);
        const float corr = epi_corr(er, c4.w, ec);
        float rho;
        const float c = epi_code(x, c4.x, fmaf(corr, c4.x, 0.5f), ec, rho);
        const bool near = fabsf(rho) > re.rho_lim;
        float k = epi_key(x, -corr, c, re.zb, c4, ec);
        if (near) {
            const float c2 = fminf(fmaxf(c + (rho > 0.0f ? 1.0f : -1.0f), -ec.ls), ec.ls);
            k = fminf(k, epi_key(x, -corr, c2, re.zb, c4, ec));
        }
        if (!(k < fminf(L.key[kListK - 1], L.tw))) continue;
        if (c == 0.0f && !near) {
            if (L.has_zero) continue;
            L.has_zero = 1;  // later s-code-0 keys carry the penalty in the main pass
        }
        const int q = j >> 3;
        const int d = q == 0 ? od[0] : (q == 1 ? od[1] : (q == 2 ? od[2] : od[3]));
        // a clean key (code not near a boundary, offset not clamped) is an
        // upper bound of the residual up to beta: it may tighten the window,
        // and the re-score may bound the best residual with it
        bool clean = false;
        if (!near) {
            const float ostar = (re.Sb - c * c4.w * ec.inv4ls) * ec.invm;
            clean = ostar < ec.pmax;
        }
        list_insert(L, k, (uint32_t)(d * 8 + (j & 7)) | (clean ? kCleanBit : 0u));
        if (clean && k < L.T) list_adopt(L, k, re, ec);
    }
}

// Symmetry source map (output (y,x) reads input (sy,sx)), n x n block.
__device__ __forceinline__ void sym_src(int k, int n, int y, int x, int &sy, int &sx)
{
    switch (k) {
    case 0: sy = y; sx = x; break;
    case 1: sy = n - 1 - x; sx = y; break;
    case 2: sy = n - 1 - y; sx = n - 1 - x; break;
    case 3: sy = x; sx = n - 1 - y; break;
    case 4: sy = y; sx = n - 1 - x; break;
    case 5: sy = n - 1 - y; sx = x; break;
    case 6: sy = x; sx = y; break;
    default: sy = n - 1 - x; sx = n - 1 - y; break;
    }
}

// The same map without branches, for threads whose symmetries differ: with
// (u, v) = (x, y) when S_k swaps the axes, else (y, x), the source pixel is
// (u ^ my, v ^ mx), where my, mx are 0 or n-1 (n a power of two, so n-1-u =
// u ^ (n-1)).  Bit k of 0xCA: axes swapped; of 0xA6: rows flipped; of 0x9C:
// columns flipped (k numbered as in sym_src).
struct SymFlags {
    int swap, my, mx;
};

__device__ __forceinline__ SymFlags sym_flags(int k, int n)
{
    return SymFlags{(0xCA >> k) & 1, ((0xA6 >> k) & 1) * (n - 1), ((0x9C >> k) & 1) * (n - 1)};
}

__device__ __forceinline__ int sym_src_index(const SymFlags &f, int ln, int y, int x)
{
    const int u = f.swap ? x : y, v = f.swap ? y : x;
    return ((u ^ f.my) << ln) + (v ^ f.mx);
}

// Compaction of the search dimensions: ranges that need screening (all but
// shadow ranges) and domains that need screening (all but flat domains), in
// their original order.  counts[0] = ranges kept, counts[1] = first shadow
// range, counts[2] = domains kept, counts[3] = first flat domain (-1: none).
struct CompactBufs {
    int *rkeep, *dkeep;   // flags
    int *act;             // kept range ids (search row j -> range act[j])
    int *dact;            // kept domain ids
    int *counts;          // 4 ints, see above
    float4 *dconst_c;     // epilogue constants of the kept domains, in order
    int *dmap;            // kept domain j -> original domain id
    uint4 *bmask;         // per statistics block: keep flags of its items (bit i of word i / 32)
    int *bcount;          // per statistics block: kept items
};
// Device buffers of one encode (sub-buffers of its workspace).
struct EncBufs {
    RangeInfo *ri;
    DomainInfo *di;
    float4 *dconst;
    uint16_t *bblk, *qblk;
    float *rs32, *cb32;
    __half *ra16, *cb16;
    ListEntry *lists;
    uint32_t *winner;
    long long *winx;      // the winner's exact cross term (kNoCross where unknown)
    int *fb_list, *fb_count, *err, *tbest;
    void *partial, *span;
    CompactBufs cb;
};

// One slice of a batched encode: everything its kernels need, read by the
// batched launches from a device array indexed by the slice (the last grid
// dimension).  abase/bbase: first rows of the slice's operands in the
// batch's shared operand buffers (tensor-core search).
constexpr int kMaxBatch = 1024;  // slices in one batched encode

struct SliceCtx {
    Geometry g;
    EpiConst ec;
    EncBufs b;
    const void *img;
    fic_map *maps;
    int n_split, n_lists, target;
    int rb, db;  // range and domain blocks of the statistics and operand-row kernels
    int abase, bbase;
    int r_begin;  // ranges of the slices before this one (context order)
};

// Number of candidate-dimension splits actually used: enough work items for
// about `target` (a few waves over the SMs) given the number of row tiles
// that have ranges to screen, capped by the list layout (max_split) and by
// a minimum number of candidate tiles per split (so that a work item
// amortises its setup and its lists see enough candidates to tighten; the
// persistent tensor-core search, recognised by its column tile, only: the
// FP32 search launches one short CTA per item and wants the items).  A
// tensor-core tile of 16x16 ranges (m = 256) is four times the MMA and copy
// work of one of 8x8 ranges, and the level of a quadtree that uses it has few
// ranges: there one tile per split suffices.
constexpr int kMinSplitTiles = 6;  // tensor-core super-tiles of 192 columns
__host__ __device__ __forceinline__ int active_splits(int row_tiles, int col_tiles, int target, int max_split,
                                                     int col_tile, int m)
{
    if (row_tiles <= 0 || col_tiles <= 0) return 1;
    int s = target / row_tiles;
    s = s < 1 ? 1 : s;
    s = s > max_split ? max_split : s;
    const int by_tiles = col_tile == 192 ? col_tiles / (m >= 256 ? 1 : kMinSplitTiles) : col_tiles;
    s = s > by_tiles ? by_tiles : s;
    return s < 1 ? 1 : s;
}

// First candidate tile of split s of ns over `tiles` tiles.  The tensor-core
// search (column unit 192) takes its items split-major from a queue shared by
// all CTAs, so its splits shrink from 1.5x to 0.5x the mean size (boundary
// tiles * (3 s ns - s^2) / (2 ns^2)): the items that start last are short
// and the SMs run out of work together.  The FP32 search's splits are equal.
__host__ __device__ __forceinline__ int split_tile(int tiles, int s, int ns, int col_tile)
{
    if (col_tile != 192) return (int)((long long)tiles * s / ns);
    return (int)((long long)tiles * (3LL * s * ns - (long long)s * s) / (2LL * ns * ns));
}

// ---------------------------------------------------------------- launches
// (host-side wrappers, each returns cudaError_t of the launch)
cudaError_t launch_search_simt(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                               const DomainInfo *di, const CompactBufs &cb, int dense, const float *rs32,
                               const float *cb32, ListEntry *lists, int max_split, int target, int *tbest,
                               float *dump, cudaStream_t st);
// Wall-clock limit of each bounded pipeline wait of the tensor-core search
// (2 s unless set; the drain at exit always allows 2 s).
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;
unsigned long long wait_limit_ns();
void set_wait_limit_ns(unsigned long long ns);  // 0: the default
bool search_tc_supported(const Geometry &g);
size_t search_tc_smem(const Geometry &g);
int search_tc_tile();
int search_tc_lists_per_split();
int search_tc_rows(int rows);  // range operand rows allocated (multiple of the TMA box)
int search_tc_cols(int cols);  // candidate operand rows allocated (multiple of the tile)
cudaError_t launch_search_tc(const Geometry &g, const EpiConst &ec, const RangeInfo *ri, const CompactBufs &cb,
                             int dense, const __half *ra16, const __half *cb16, ListEntry *lists, int max_split,
                             int target, int *tbest, float *dump, int *err, int *queue, cudaStream_t st);
int search_simt_lists_per_split();
// Batched encode of n slices (ctx: device array of their contexts), one
// launch per stage over the slices (the per-slice stages: once per group of
// equal slices).
int stats_grid(const Geometry &g);  // blocks of the statistics launch of one slice
cudaError_t launch_stats_batch(const Geometry &g, const SliceCtx *ctx, int n, int blocks, int dense, int tc_mode,
                               cudaStream_t st);
cudaError_t launch_compact_seed_batch(const SliceCtx *ctx, int n, int ranges, int m, cudaStream_t st);
cudaError_t launch_rows_batch(const Geometry &g, const SliceCtx *ctx, int n, int blocks, cudaStream_t st);
cudaError_t launch_search_tc_batch(const Geometry &g, const __half *ra16, int arows, const __half *cb16, int brows,
                                   const SliceCtx *ctx, int n, int dense, int *queue, cudaStream_t st);
cudaError_t launch_search_simt_batch(const SliceCtx *ctx, int n, int max_ranges, int max_split, int dense,
                                     cudaStream_t st);
cudaError_t launch_rescore_batch(const SliceCtx *ctx, int n, int total_ranges, bool any_wide, bool any_narrow,
                                 int max_m, int lists_per_split, int col_tile, int exact_scan, int n_sm,
                                 cudaStream_t st);
cudaError_t launch_finalize_batch(const SliceCtx *ctx, int n, int ranges, bool wide, cudaStream_t st);
cudaError_t launch_rescore(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                           const DomainInfo *di, const uint16_t *bblk, const uint16_t *qblk,
                           const ListEntry *lists, int max_lists, const int *counts, const int *act,
                           const int *rkeep, int lists_per_split, int col_tile, int target, int max_split, int n_sm,
                           int exact_scan, uint32_t *winner, long long *winx, int *fb_list, int *fb_count,
                           void *partial, void *span, cudaStream_t st);
size_t span_bytes(const Geometry &g, int max_lists);
// The exact scans of the ranges the re-score queued and the map output, one
// launch.
cudaError_t launch_scans_finalize(const Geometry &g, const RangeInfo *ri, const DomainInfo *di, const uint16_t *bblk,
                                  const uint16_t *qblk, const int *fb_list, int *fb_count, void *partial,
                                  const int *counts, const int *dmap, int col_tile, int target, int max_split,
                                  int lists_per_split, int max_lists, void *span, uint32_t *winner,
                                  const long long *winx, const int *err, fic_map *maps, const EpiConst &ec,
                                  const float4 *dconst, int n_sm, cudaStream_t st);
size_t fallback_partial_bytes(const Geometry &g);
size_t decode_workspace_bytes(const Geometry &g);
cudaError_t launch_decode(const Geometry &g, const fic_map *maps, float init, int iters, void *ws,
                          float *out, cudaStream_t st);
// Per-thread epilogue constants of range r.
__device__ __forceinline__ RangeEpi range_epi(const RangeInfo &ri, const EpiConst &ec)
{
    RangeEpi re;
    re.zb = ri.zb;
    re.rho_lim = ri.rho_lim;
    re.sbbc = ri.sbbc;
    re.sqrt_sbbc = sqrtf(fmaxf(ri.sbbc, 0.0f));
    re.bA = ri.beta_a;
    re.bQ = ri.beta_q;
    re.Sb = (float)ri.Sb;
    re.shadow = ri.shadow;
    return re;
}
cudaError_t launch_prep(const Geometry &g, const void *img, const EpiConst &ec, int dense, int tc_mode,
                        const int *active,
                        RangeInfo *ri, DomainInfo *di, float4 *dconst, uint16_t *bblk, uint16_t *qblk, float *rs32,
                        float *cb32, __half *ra16, __half *cb16, int *tbest, const CompactBufs &cb, int *zero4,
                        int seed, cudaStream_t st);
// The encode pipeline on a caller-provided device workspace (never allocates).
int encode_with_workspace(const void *img, int w, int h, int pitch_px, const fic_params *p, fic_map *maps,
                          int maps_cap, int *n_maps, void *workspace, size_t workspace_bytes, void *stream);
// Levels of an adaptive quadtree encode (device arrays per level).
constexpr int kMaxLevels = 3;  // range sizes 16, 8, 4
struct QtLevels {
    int levels;
    int R[kMaxLevels], nx[kMaxLevels], n[kMaxLevels];
    const int *active[kMaxLevels];
    const int *leaf[kMaxLevels];
    const fic_map *maps[kMaxLevels];
    int list_off[kMaxLevels];  // offset of level l's leaf list in the lists buffer
};
cudaError_t launch_qt_split(int R, int nx, int m, const fic_map *maps, const int *active, double rms_split, int last,
                            int *leaf, int *active_next, cudaStream_t st);
cudaError_t launch_qt_gather(const QtLevels &lv, int *lists, fic_qmap *out, int cap, int *counts, cudaStream_t st);
// Differentiable refinement (the unrolled decoder with FP32 s, o and its adjoint).
struct RefineGeo {
    int w, h, n, ln, nx, R, t, U, V, D;
};
struct RefineBufs {
    int *roff, *rsym;                 // per range: domain offset, symmetry
    int *dcount, *doff, *cursor, *drng;  // domain -> ranges index (CSR, rows sorted)
    float *tmp, *g[2];                // scratch iterate, adjoint ping-pong
    double *partial;                  // loss partial sums
    int *step;                        // Adam step counter (device)
    float *ds, *dof, *m, *v;          // gradients, Adam moments (2R)
    float *C;                         // per-domain adjoint sums [D][m]
    int *nitem, *ioff;                // adjoint work items per domain, offsets (D + 1)
    int4 *items;                      // (domain, first user, end user) per item, at most R
    float *ipart;                     // per-item partial sums [R][m]
};
cudaError_t refine_ranges(const RefineGeo &rg, const fic_map *maps, const RefineBufs &b, bool with_index,
                          cudaStream_t st);
cudaError_t refine_forward(const RefineGeo &rg, const RefineBufs &b, const float *s, const float *o, float init,
                           int iters, float *ckpt, float *x_out, cudaStream_t st);
cudaError_t refine_backward(const RefineGeo &rg, const RefineBufs &b, const float *s, const float *o, int iters,
                            const float *ckpt, const float *grad_x, float *ds, float *dof, cudaStream_t st);
cudaError_t refine_loss(const RefineGeo &rg, const RefineBufs &b, const float *x, const void *img, int B, int pitch,
                        float *g, float *loss, int advance, cudaStream_t st);
cudaError_t refine_adam(const RefineGeo &rg, const RefineBufs &b, float *s, float *o, float lr, float P,
                        cudaStream_t st);
size_t refine_partials(const RefineGeo &rg);
// Key-space value that excludes s-code-0 candidates once a list holds one.
constexpr float kZeroPenalty = 1e30f;

}  // namespace fic
