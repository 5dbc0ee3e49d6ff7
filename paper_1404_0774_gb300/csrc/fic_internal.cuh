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
#include <cuda_runtime.h>
#include <stdint.h>

#include "fic.h"

namespace fic {

constexpr int kListK = 4;          // entries per candidate list
constexpr int kMaxM = 256;         // largest range (16 x 16)
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: x + kMagic rounds x to an integer

struct Geometry {
    int w, h, pitch;   // image size and row pitch (elements)
    int n, t, m;       // range size, domain stride, pixels per range
    int nx, ny, R;     // ranges per row / column / total
    int U, V, D;       // domains per row / column / total
    int N;             // candidates = 8*D
    int B, P;          // bit depth, 2^B - 1
    int s_bits, o_bits, Ls, Lo;
    int split_hilo;    // 1 when q' must be split into two exact FP16 parts
    int KP;            // FP16 operand row length (tensor-core layout)
    int mod_g;         // 1 when G is an integer (z may be reduced mod G)
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

// Code decision of one candidate: returns c (integer-valued float) and rho.
__device__ __forceinline__ float epi_code(float X, float alpha, const EpiConst &ec, float &rho)
{
    const float u = __saturatef(fmaf(X, alpha, 0.5f));
    const float r = fmaf(u, ec.two_ls, -ec.ls);  // Ls * clamp(s, -1, 1)
    const float c = __fsub_rn(__fadd_rn(r, kMagic), kMagic);
    rho = __fsub_rn(r, c);
    return c;
}

// Screening key for a fixed code c.
__device__ __forceinline__ float epi_key(float X, float c, float zb, float4 dc, const EpiConst &ec)
{
    const float z = fmaf(c, -dc.y, zb);
    const float e = __fsub_rn(fmaf(z, ec.invG, kMagic), kMagic);
    const float wv = fmaf(e, -ec.G, z);
    const float y = fmaf(c, dc.z, -X);
    const float cy = __fmul_rn(c, y);
    return fmaf(__fmul_rn(wv, ec.lambda), wv, cy);
}

// Main pass over 32 consecutive candidates (4 domains x 8 symmetries):
// X[] (cross terms) is overwritten by the keys.  Branch-free.  Returns whether
// this thread needs the rare pass: a key below `thr`, or a code decided next
// to its rounding boundary.  Lanes beyond the ragged end carry X = NaN (their
// keys are NaN and compare false everywhere).
// zpen: added to the key of s-code-0 candidates (their residual is one value
// per range; once the list holds one, the others need never be looked at).
__device__ __forceinline__ bool epi_keys32(float (&X)[32], const float4 (&dc)[4], float zb, float rho_lim,
                                           const EpiConst &ec, float thr, float zpen)
{
    float kmin = __int_as_float(0x7f800000);
    float rmax = 0.0f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const float4 c4 = dc[j >> 3];
        float rho;
        const float c = epi_code(X[j], c4.x, ec, rho);
        const float zero = __saturatef(fmaf(c, -c, 1.0f));  // 1 for c = 0, else 0 (c is an integer)
        const float k = fmaf(zero, zpen, epi_key(X[j], c, zb, c4, ec));
        X[j] = k;
        kmin = fminf(kmin, k);
        rmax = fmaxf(rmax, fabsf(rho));
    }
    return kmin < thr || rmax > rho_lim;
}

__device__ __forceinline__ float4 pick4(const float4 (&dc)[4], int q)
{
    return q == 0 ? dc[0] : (q == 1 ? dc[1] : (q == 2 ? dc[2] : dc[3]));
}

// Rare pass for one thread: keys and cross terms staged in shared memory at
// krow[j*stride], xrow[j*xstride].  Handles codes next to a rounding boundary
// (the key becomes the smaller of the two neighbouring codes' keys: a lower
// bound of the residual FP64 decides) and list insertion with s-code-0
// de-duplication (all such candidates of a range have one residual).
static __device__ __noinline__ void epi_rare(const float *krow, int stride, const float *xrow, int xstride,
                                      uint32_t idx0, const float4 (&dc)[4], const RangeEpi &re,
                                      const EpiConst &ec, ListState &L, int nvalid)
{
#pragma unroll 1
    for (int j = 0; j < nvalid; ++j) {
        float k = krow[j * stride];
        const float x = xrow[j * xstride];
        const float4 c4 = pick4(dc, j >> 3);
        float rho;
        const float c = epi_code(x, c4.x, ec, rho);
        const bool near = fabsf(rho) > re.rho_lim;
        if (near) {
            const float c2 = fminf(fmaxf(c + (rho > 0.0f ? 1.0f : -1.0f), -ec.ls), ec.ls);
            k = fminf(k, epi_key(x, c2, re.zb, c4, ec));
        }
        if (!(k < fminf(L.key[kListK - 1], L.tw))) continue;
        if (c == 0.0f && !near) {
            if (L.has_zero) continue;
            L.has_zero = 1;  // later s-code-0 keys carry the penalty in the main pass
        }
        list_insert(L, k, idx0 + j);
        if (k < L.T && !near) {
            // a clean key (code not near a boundary, offset not clamped) is an
            // upper bound of the residual up to beta: it may tighten the window
            const float ostar = (re.Sb - c * c4.w * ec.inv4ls) * ec.invm;
            if (ostar < ec.pmax) list_adopt(L, k, re, ec);
        }
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

__device__ __forceinline__ int load_px(const void *img, int B, size_t off)
{
    return B <= 8 ? (int)((const uint8_t *)img)[off] : (int)((const uint16_t *)img)[off];
}

// ---------------------------------------------------------------- launches
// (host-side wrappers, each returns cudaError_t of the launch)
cudaError_t launch_search_simt(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                               const DomainInfo *di, const float4 *dconst, const float *rs32,
                               const float *cb32, ListEntry *lists, int n_split, int *tbest, float *dump,
                               cudaStream_t st);
bool search_tc_supported(const Geometry &g);
size_t search_tc_smem(const Geometry &g);
int search_tc_tile();
int search_tc_rows(int rows);  // operand rows allocated (multiple of the TMA box)
cudaError_t launch_search_tc(const Geometry &g, const EpiConst &ec, const RangeInfo *ri, const float4 *dconst,
                             const __half *ra16, const __half *cb16, ListEntry *lists, int n_split, int *tbest,
                             float *dump, int *err, cudaStream_t st);
int search_simt_lists_per_split();
cudaError_t launch_rescore(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                           const DomainInfo *di, const uint16_t *bblk, const uint16_t *qblk,
                           const ListEntry *lists, int n_lists, uint32_t *winner, int *fb_list,
                           int *fb_count, cudaStream_t st);
size_t fallback_partial_bytes(const Geometry &g);
cudaError_t launch_fallback(const Geometry &g, const RangeInfo *ri, const DomainInfo *di,
                            const uint16_t *bblk, const uint16_t *qblk, const int *fb_list,
                            const int *fb_count, void *partial, uint32_t *winner, cudaStream_t st);
cudaError_t launch_finalize(const Geometry &g, const RangeInfo *ri, const DomainInfo *di,
                            const uint16_t *bblk, const uint16_t *qblk, const uint32_t *winner,
                            const int *err, fic_map *maps, cudaStream_t st);
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
cudaError_t launch_prep(const Geometry &g, const void *img, const EpiConst &ec, RangeInfo *ri, DomainInfo *di,
                        float4 *dconst, uint16_t *bblk, uint16_t *qblk, float *rs32, float *cb32,
                        __half *ra16, __half *cb16, int *tbest, cudaStream_t st);
cudaError_t launch_seed(const Geometry &g, const EpiConst &ec, const RangeInfo *ri, const DomainInfo *di,
                        const float4 *dconst, const uint16_t *bblk, const uint16_t *qblk, int *tbest,
                        cudaStream_t st);
// The encode pipeline on a caller-provided device workspace (never allocates).
int encode_with_workspace(const void *img, int w, int h, int pitch_px, const fic_params *p, fic_map *maps,
                          int maps_cap, int *n_maps, void *workspace, size_t workspace_bytes, void *stream);
// Key-space value that excludes s-code-0 candidates once a list holds one.
constexpr float kZeroPenalty = 1e30f;

}  // namespace fic
