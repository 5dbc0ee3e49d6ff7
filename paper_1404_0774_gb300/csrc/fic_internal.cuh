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
//   w: g     = sqrt(m/den) (0 for a flat domain): |Xt|*g = sqrt(explained variance)
struct EpiConst {
    float two_ls, ls;
    float G, invG;
    float lambda;
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
};

__device__ __forceinline__ void list_init(ListState &L)
{
#pragma unroll
    for (int i = 0; i < kListK; ++i) {
        L.key[i] = __int_as_float(0x7f800000);  // +inf
        L.idx[i] = 0xffffffffu;
    }
    L.has_zero = 0;
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

// Process 32 consecutive candidates idx0..idx0+31 (4 domains x 8 symmetries)
// of one range.  X[] holds Xt per candidate and is overwritten by the keys.
// Only the first `nvalid` candidates are real (a ragged tail of the
// candidate dimension); the rest get an infinite key.
__device__ __forceinline__ void epi_chunk32(float (&X)[32], uint32_t idx0, const float4 (&dc)[4],
                                            float zb, float rho_lim, const EpiConst &ec,
                                            ListState &L, int nvalid = 32)
{
    float kmin = __int_as_float(0x7f800000);
    float rmax = 0.0f;
    float xs[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const float4 c4 = dc[j >> 3];
        float rho;
        const float c = epi_code(X[j], c4.x, ec, rho);
        xs[j] = X[j];
        float k = epi_key(X[j], c, zb, c4, ec);
        if (j >= nvalid) {
            k = __int_as_float(0x7f800000);
            rho = 0.0f;
        }
        rmax = fmaxf(rmax, fabsf(rho));
        X[j] = k;
        kmin = fminf(kmin, k);
    }
    if (rmax > rho_lim) {
        // near a rounding boundary of s: the code FP64 picks may be the other
        // neighbour, so rank by the smaller of the two keys
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float4 c4 = dc[j >> 3];
            float rho;
            const float c = epi_code(xs[j], c4.x, ec, rho);
            if (j < nvalid && fabsf(rho) > rho_lim) {
                float c2 = c + (rho > 0.0f ? 1.0f : -1.0f);
                c2 = fminf(fmaxf(c2, -ec.ls), ec.ls);
                const float k2 = epi_key(xs[j], c2, zb, c4, ec);
                X[j] = fminf(X[j], k2);
                kmin = fminf(kmin, X[j]);
            }
        }
    }
    if (kmin < L.key[kListK - 1]) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            float kj = X[j];
            if (kj < L.key[kListK - 1]) {
                float rho;
                const float c = epi_code(xs[j], dc[j >> 3].x, ec, rho);
                if (c == 0.0f && fabsf(rho) <= rho_lim) {
                    // every s-code-0 candidate of a range has the same residual
                    // (Sbb_c plus the offset term): keep only the first
                    if (L.has_zero) continue;
                    L.has_zero = 1;
                }
                list_insert(L, kj, idx0 + j);
            }
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
cudaError_t launch_prep(const Geometry &g, const void *img, RangeInfo *ri, DomainInfo *di,
                        float4 *dconst, uint16_t *bblk, uint16_t *qblk, float *rs32, float *cb32,
                        __half *ra16, __half *cb16, cudaStream_t st);
cudaError_t launch_search_simt(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                               const DomainInfo *di, const float4 *dconst, const float *rs32,
                               const float *cb32, ListEntry *lists, int n_split, float *dump,
                               cudaStream_t st);
bool search_tc_supported(const Geometry &g);
size_t search_tc_smem(const Geometry &g);
int search_tc_tile();
int search_tc_rows(int rows);  // operand rows allocated (multiple of the TMA box)
cudaError_t launch_search_tc(const Geometry &g, const EpiConst &ec, const RangeInfo *ri, const float4 *dconst,
                             const __half *ra16, const __half *cb16, ListEntry *lists, int n_split, float *dump,
                             int *err, cudaStream_t st);
int search_simt_lists_per_split();
cudaError_t launch_rescore(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                           const DomainInfo *di, const uint16_t *bblk, const uint16_t *qblk,
                           const ListEntry *lists, int n_lists, const float *qp2max, uint32_t *winner,
                           int *fb_list, int *fb_count, cudaStream_t st);
cudaError_t launch_fallback(const Geometry &g, const RangeInfo *ri, const DomainInfo *di,
                            const uint16_t *bblk, const uint16_t *qblk, const int *fb_list,
                            const int *fb_count, uint32_t *winner, cudaStream_t st);
cudaError_t launch_finalize(const Geometry &g, const RangeInfo *ri, const DomainInfo *di,
                            const uint16_t *bblk, const uint16_t *qblk, const uint32_t *winner,
                            const int *err, fic_map *maps, cudaStream_t st);
size_t decode_workspace_bytes(const Geometry &g);
cudaError_t launch_decode(const Geometry &g, const fic_map *maps, float init, int iters, void *ws,
                          float *out, cudaStream_t st);
cudaError_t launch_qp2max(const Geometry &g, const DomainInfo *di, float *qp2max, cudaStream_t st);

}  // namespace fic
