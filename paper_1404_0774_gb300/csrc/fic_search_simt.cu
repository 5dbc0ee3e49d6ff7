// Plain FP32 CUDA-core range-domain search (the speedup baseline).
//
// Same problem as the tensor-core search: for every range (Algorithm 3's
// "one thread per range block") and every candidate 8d+k, the cross term
// Xt = sum q'b' - e_r f_d/m is formed in FP32 on the CUDA cores, then the
// shared FP32 screening epilogue (eq 8-12 with quantisation) keeps each
// range's best candidates.  A CTA owns 128 ranges and streams a contiguous
// slice of the candidate dimension in tiles of 64; the 128 x 64 cross terms
// are computed with an 8 x 4 register tile per thread and staged through
// shared memory for the epilogue (two threads per range, 32 candidates each).
#include "fic_internal.cuh"

namespace fic {

namespace {
constexpr int BM = 128;  // ranges per CTA
constexpr int BN = 64;   // candidates per tile
constexpr int KC = 64;   // pixels per k chunk
constexpr int XS = BN + 1;
}  // namespace

__device__ __forceinline__ void search_simt_cta(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                                                const DomainInfo *di, const float4 *dconst, const int *act,
                                                const int *dmap, const int *counts, int dense, const float *rs32,
                                                const float *cb32, ListEntry *lists, int max_split, int target,
                                                int *tbest, float *dump, int bx, int by)
{
    extern __shared__ float smem[];
    float *As = smem;              // [KC][BM]
    float *Bs = As + KC * BM;      // [KC][BN]
    float *Xs = Bs + KC * BN;      // [BM][XS]
    __shared__ float er_s[BM];
    __shared__ float fdm_s[BN];

    const int tid = threadIdx.x;
    // rows are the ranges kept for screening, columns the candidates of the
    // kept domains (both compacted, in original order)
    const int nrow = counts[0];
    const int ncol = 8 * counts[2];
    const int r0 = bx * BM;
    const int split = by;
    // contiguous slice of the candidate dimension, in whole tiles
    const int tiles = (ncol + BN - 1) / BN;
    const int n_split = active_splits((nrow + BM - 1) / BM, tiles, target, max_split, BN, g.m);
    if (r0 >= nrow || split >= n_split) return;  // CTA-uniform: nothing to screen
    const int t_begin = (int)((long long)tiles * split / n_split);
    const int t_end = (int)((long long)tiles * (split + 1) / n_split);

    if (tid < BM) er_s[tid] = (r0 + tid < nrow) ? (float)ri[act[r0 + tid]].e_r : 0.0f;

    // epilogue role: one range row, one half of the tile
    const int er_row = tid & (BM - 1);
    const int er_half = tid >> 7;
    const bool row_live = r0 + er_row < nrow;
    const int my_r = row_live ? act[r0 + er_row] : 0;  // range id
    RangeEpi re{};
    if (row_live) re = range_epi(ri[my_r], ec);
    const bool scr = row_live && (dense || !re.shadow);
    ListState L;
    list_init(L);

    // compute role: 8 ranges x 4 candidates
    const int tr = tid >> 4, tc = tid & 15;

    for (int tile = t_begin; tile < t_end; ++tile) {
        const int n0 = tile * BN;
        float acc[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;

        for (int k0 = 0; k0 < g.m; k0 += KC) {
            __syncthreads();
            // ranges: As[k][r] = b'(r0 + r, k0 + k)
            for (int f = tid; f < BM * (KC / 4); f += 256) {
                const int r = f % BM, k4 = f / BM;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (r0 + r < nrow && k0 + 4 * k4 < g.m)
                    v = *reinterpret_cast<const float4 *>(rs32 + (size_t)(r0 + r) * g.m + k0 + 4 * k4);
                As[(4 * k4 + 0) * BM + r] = v.x;
                As[(4 * k4 + 1) * BM + r] = v.y;
                As[(4 * k4 + 2) * BM + r] = v.z;
                As[(4 * k4 + 3) * BM + r] = v.w;
            }
            // candidates: Bs[k][c] = q'(n0 + c, k0 + k)
            for (int f = tid; f < BN * (KC / 4); f += 256) {
                const int c = f % BN, k4 = f / BN;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (n0 + c < ncol && k0 + 4 * k4 < g.m)
                    v = *reinterpret_cast<const float4 *>(cb32 + (size_t)(n0 + c) * g.m + k0 + 4 * k4);
                Bs[(4 * k4 + 0) * BN + c] = v.x;
                Bs[(4 * k4 + 1) * BN + c] = v.y;
                Bs[(4 * k4 + 2) * BN + c] = v.z;
                Bs[(4 * k4 + 3) * BN + c] = v.w;
            }
            if (k0 == 0 && tid < BN)
                fdm_s[tid] = (n0 + tid < ncol) ? (float)di[dmap[(n0 + tid) >> 3]].f_d / (float)g.m : 0.0f;
            __syncthreads();
            const int kn = min(KC, g.m - k0);
#pragma unroll 4
            for (int k = 0; k < kn; ++k) {
                const float4 a0 = *reinterpret_cast<const float4 *>(As + k * BM + tr * 8);
                const float4 a1 = *reinterpret_cast<const float4 *>(As + k * BM + tr * 8 + 4);
                const float4 b = *reinterpret_cast<const float4 *>(Bs + k * BN + tc * 4);
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
            }
        }
        // Xt = sum q'b' - e_r f_d / m
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                Xs[(tr * 8 + i) * XS + tc * 4 + j] =
                    fmaf(-er_s[tr * 8 + i], fdm_s[tc * 4 + j], acc[i][j]);
        __syncthreads();
        if (row_live && dump) {
            const int c0 = n0 + er_half * 32;
            for (int j = 0; j < 32 && c0 + j < ncol; ++j)
                dump[(size_t)my_r * g.N + dmap[(c0 + j) >> 3] * 8 + (j & 7)] = Xs[er_row * XS + er_half * 32 + j];
        } else if (scr) {
            const float Tg = ord2f(__ldcg(tbest + my_r));  // best key other CTAs found
            list_adopt(L, Tg, re, ec);
            L.Tpub = fminf(L.Tpub, Tg);
            const int c0 = n0 + er_half * 32;
            const int nvalid = min(32, ncol - c0);
            if (nvalid > 0) {
                const float *xrow = Xs + er_row * XS + er_half * 32;
                float X[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) X[j] = j < nvalid ? xrow[j] : __int_as_float(0x7fc00000);
                float4 dc[4];
                int od[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int jd = (c0 >> 3) + q;
                    const bool ok = jd < counts[2];
                    dc[q] = ok ? dconst[jd] : make_float4(0.f, 0.f, 0.f, 0.f);
                    od[q] = ok ? dmap[jd] : 0;
                }
                const uint32_t mask = epi_keys32(X, dc, re.zb, re.rho_lim, 0.0f, ec, fminf(L.key[kListK - 1], L.tw),
                                                 L.has_zero ? kZeroPenalty : 0.0f);
                if (mask) {
                    epi_rare(xrow, 1, od, dc, 0.0f, re, ec, L, mask);
                    if (L.T < L.Tpub) {
                        atomicMin(tbest + my_r, f2ord(L.T));
                        L.Tpub = L.T;
                    }
                }
            }
        }
    }
    if (scr && !dump) {
        ListEntry *dst = lists + ((size_t)my_r * max_split * 2 + split * 2 + er_half) * kListK;
#pragma unroll
        for (int i = 0; i < kListK; ++i) dst[i] = ListEntry{L.key[i], L.idx[i]};
    }
}

__global__ void __launch_bounds__(256) k_search_simt(Geometry g, EpiConst ec, const RangeInfo *ri,
                                                     const DomainInfo *di, const float4 *dconst,
                                                     const int *act, const int *dmap, const int *counts,
                                                     int dense, const float *rs32, const float *cb32,
                                                     ListEntry *lists, int max_split, int target, int *tbest,
                                                     float *dump)
{
    grid_dep_sync();
    search_simt_cta(g, ec, ri, di, dconst, act, dmap, counts, dense, rs32, cb32, lists, max_split, target, tbest, dump,
                    blockIdx.x, blockIdx.y);
}

// Batched: blockIdx.z = slice.
__global__ void __launch_bounds__(256) k_search_simt_batch(const SliceCtx *__restrict__ ctx, int dense)
{
    grid_dep_sync();
    const SliceCtx c = ctx[blockIdx.z];
    if ((int)blockIdx.y >= c.n_split || (int)blockIdx.x * BM >= c.g.R) return;  // CTA-uniform
    const EncBufs &b = c.b;
    search_simt_cta(c.g, c.ec, b.ri, b.di, b.cb.dconst_c, b.cb.act, b.cb.dmap, b.cb.counts, dense, b.rs32, b.cb32,
                    b.lists, c.n_split, c.target, b.tbest, nullptr, blockIdx.x, blockIdx.y);
}

int search_simt_lists_per_split() { return 2; }

cudaError_t launch_search_simt(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                               const DomainInfo *di, const CompactBufs &cb, int dense, const float *rs32,
                               const float *cb32, ListEntry *lists, int max_split, int target, int *tbest,
                               float *dump, cudaStream_t st)
{
    const size_t smem = sizeof(float) * (KC * BM + KC * BN + BM * XS);
    cudaError_t e = cudaFuncSetAttribute(k_search_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.R + BM - 1) / BM, max_split);
    return launch_dep(k_search_simt, grid, dim3(256), smem, st, g, ec, ri, di, (const float4 *)cb.dconst_c,
                      (const int *)cb.act, (const int *)cb.dmap, (const int *)cb.counts, dense, rs32, cb32, lists,
                      max_split, target, tbest, dump);
}

cudaError_t launch_search_simt_batch(const SliceCtx *ctx, int n, int max_ranges, int max_split, int dense,
                                     cudaStream_t st)
{
    const size_t smem = sizeof(float) * (KC * BM + KC * BN + BM * XS);
    cudaError_t e = cudaFuncSetAttribute(k_search_simt_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_dep(k_search_simt_batch, dim3((max_ranges + BM - 1) / BM, max_split, n), dim3(256), smem, st, ctx,
                      dense);
}

}  // namespace fic
