// Prep kernels: range blocks and domain pool (Section V, Algorithm 1).
//
// The paper generates the codebook (every domain contracted by tau and
// expanded by the 8 symmetries) on the fly inside the per-range thread.  Here
// it is built once per image: tau(d) is computed once per domain as the 2x2
// sum q (an exact integer; the mean is q/4), its statistics once per domain
// (they are symmetry-invariant), and the 8 symmetric copies are written as
// candidate rows of the operand layouts the search kernels stream.
#include "fic_internal.cuh"

namespace fic {

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// One warp per range (lanes over pixels): statistics, centre, operand rows.
__global__ void k_range_prep(Geometry g, EpiConst ec, const void *img, RangeInfo *ri, uint16_t *bblk, int *tbest)
{
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= g.R) return;  // warp-uniform
    const int ry = (r / g.nx) * g.n, rx = (r % g.nx) * g.n;
    constexpr int PPL = kMaxM / 32;  // pixels per lane, upper bound
    int bv[PPL];
    long long Sb = 0, Sbb = 0;
    int bmin = 1 << 30, bmax = -1;
#pragma unroll
    for (int j = 0; j < PPL; ++j) {
        const int i = lane + 32 * j;
        bv[j] = 0;
        if (i < g.m) {
            const int b = load_px(img, g.B, (size_t)(ry + i / g.n) * g.pitch + rx + i % g.n);
            bv[j] = b;
            Sb += b;
            Sbb += (long long)b * b;
            bmin = min(bmin, b);
            bmax = max(bmax, b);
            bblk[(size_t)r * g.m + i] = (uint16_t)b;
        }
    }
    Sb = warp_sum_ll(Sb);
    Sbb = warp_sum_ll(Sbb);
    for (int off = 16; off > 0; off >>= 1) {
        bmin = min(bmin, __shfl_xor_sync(0xffffffffu, bmin, off));
        bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, off));
    }
    // centre: nearest integer to the mean, kept within 2048 of every pixel so
    // that b - c_r is an exact FP16 integer
    long long cr = (2 * Sb + g.m) / (2 * (long long)g.m);
    cr = max((long long)(bmax - 2048), min((long long)(bmin + 2048), cr));
    const int c_r = (int)cr;
    const int e_r = (int)(Sb - (long long)g.m * c_r);
    long long bp2i = 0;
#pragma unroll
    for (int j = 0; j < PPL; ++j) {
        const int i = lane + 32 * j;
        if (i < g.m) {
            const int bc = bv[j] - c_r;
            bp2i += (long long)bc * bc;
        }
    }
    const double bp2 = (double)warp_sum_ll(bp2i);
    if (lane != 0) return;
    // per-range constants: integer arithmetic and FP32 only (the FP64 rate of
    // this part is a small fraction of FP32)
    RangeInfo info;
    info.Sb = Sb;
    info.Sbb = Sbb;
    info.c_r = c_r;
    info.e_r = e_r;
    const float invm = 1.0f / (float)g.m;
    info.sbbc = (float)((long long)g.m * Sbb - Sb * Sb) * invm;
    const long long z = 4LL * g.Ls * Sb;
    info.zb = (float)(g.mod_g ? z % (long long)g.G : z);
    const float bp2f = (float)bp2;
    info.bp2 = bp2f;
    // FP32 error of Ls*s: ~1e-6 when the cross term is exact, plus the
    // accumulation error of high-variance pairs (grows with sum (b-c_r)^2)
    const float eta = 1e-5f + 12.0f * g.Ls * 64.0f * bp2f * 3.552713678800501e-15f;  // 2^-48
    info.rho_lim = 0.5f - fminf(eta, 0.25f);
    // Screening allowance.  A candidate within reach of the winner has
    // |c| * sqrt(sum (q-q_mean)^2) <= 4*Ls*(sqrt(Sbb_c) + sqrt(R)), R <= Eb; its
    // centred products (hi/lo split included) then sum to at most S.  Below
    // 2^23 every FP32 partial sum of integers is exact and the cross term
    // carries no error; otherwise allow 2^-15 relative.
    const float sbbc = fmaxf(info.sbbc, 0.0f);
    const float Eb = 4.0f * (sbbc + ec.delta_o);
    const float sb = sqrtf(bp2f);
    const float sqm = sqrtf((float)g.m);
    const float S = (4.0f * g.Ls * (sqrtf(sbbc) + sqrtf(Eb)) + sqm) * sb + (g.split_hilo ? 128.0f * sqm * sb : 0.0f);
    const bool exact = S < 8.0e6f;  // < 2^23 with margin
    const float gam = 3.0517578125e-05f;  // 2^-15
    info.beta_q = exact ? 0.0f : 4.0f * g.Ls * gam * sb;
    info.beta_a = 3.814697265625e-06f * 2.0f * g.Ls * (sbbc + ec.delta_o) + 1e-3f +
                  (exact ? 0.0f : gam * g.Ls * 128.0f * sqm * sb);
    info.shadow = bmin == bmax ? 1 : 0;
    info.pad = 0;
    ri[r] = info;
    tbest[r] = 0x7f800000;  // +inf in the ordered-integer encoding of floats
}

// One block of m threads per domain.
__global__ void k_domain_prep(Geometry g, const void *img, DomainInfo *di, float4 *dconst, uint16_t *qblk)
{
    __shared__ int q_s[kMaxM];
    __shared__ long long red_s[2][kMaxM / 32];
    __shared__ int cd_s, fd_s;
    __shared__ float qp2_s[kMaxM / 32];
    const int d = blockIdx.x;
    const int i = threadIdx.x;  // pixel of the contracted block (blockDim = max(m, 32))
    const int n = g.n, m = g.m;
    const bool live = i < m;
    const int dy = (d / g.U) * g.t, dx = (d % g.U) * g.t;
    const int y = live ? i / n : 0, x = live ? i % n : 0;
    const size_t o0 = (size_t)(dy + 2 * y) * g.pitch + dx + 2 * x;
    int q = 0;
    if (live) {
        q = load_px(img, g.B, o0) + load_px(img, g.B, o0 + 1) + load_px(img, g.B, o0 + g.pitch) +
            load_px(img, g.B, o0 + g.pitch + 1);
        q_s[i] = q;
        qblk[(size_t)d * m + i] = (uint16_t)q;
    }
    long long s1 = q, s2 = (long long)q * q;
    for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, off);
        s2 += __shfl_down_sync(0xffffffffu, s2, off);
    }
    const int lane = i & 31, warp = i >> 5, nw = (m + 31) / 32;
    if (lane == 0) {
        red_s[0][warp] = s1;
        red_s[1][warp] = s2;
    }
    __syncthreads();
    if (i == 0) {
        long long Sq = 0, Sqq = 0;
        for (int w = 0; w < nw; ++w) {
            Sq += red_s[0][w];
            Sqq += red_s[1][w];
        }
        const long long cd = (2 * Sq + m) / (2 * (long long)m);
        cd_s = (int)cd;
        fd_s = (int)(Sq - (long long)m * cd);
        const long long den = (long long)m * Sqq - Sq * Sq;
        DomainInfo info;
        info.Sq = Sq;
        info.Sqq = Sqq;
        info.c_d = (int)cd;
        info.f_d = fd_s;
        info.qp2 = 0.0f;
        info.pad = 0.0f;
        di[d] = info;
        // FP32 from exact integers (no FP64 on this path)
        float4 c4;
        const float denf = (float)den;
        c4.x = den > 0 ? (2.0f * m) / denf : 0.0f;
        c4.y = (float)(g.mod_g ? Sq % (long long)g.G : Sq);
        c4.z = denf / (8.0f * m * g.Ls);
        c4.w = (float)Sq;
        dconst[d] = c4;
    }
    __syncthreads();
    const int c_d = cd_s;
    // centred value of this pixel for the variance bound
    {
        const float qc = (float)(q - c_d);
        float v = live ? qc * qc : 0.0f;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) qp2_s[warp] = v;
        __syncthreads();
        if (i == 0) {
            float t = 0.0f;
            for (int w = 0; w < nw; ++w) t += qp2_s[w];
            di[d].qp2 = t;
        }
    }
}

// Stable compaction of the items whose flag is set (one block): keeps the
// original order, writes the count, and the first unset index (-1 if none).
__global__ void __launch_bounds__(1024) k_compact(int n, const int *flag, int *list, int *count, int *first_unset)
{
    __shared__ int cnt_s[1024];
    __shared__ int first_s[32];
    const int t = threadIdx.x;
    const int seg = (n + 1023) / 1024;
    const int lo = min(n, t * seg), hi = min(n, lo + seg);
    int c = 0, fu = 0x7fffffff;
    for (int i = lo; i < hi; ++i) {
        if (flag[i]) ++c;
        else fu = min(fu, i);
    }
    cnt_s[t] = c;
    for (int off = 16; off > 0; off >>= 1) fu = min(fu, __shfl_xor_sync(0xffffffffu, fu, off));
    if ((t & 31) == 0) first_s[t >> 5] = fu;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // inclusive scan (Hillis-Steele)
        const int v = t >= off ? cnt_s[t - off] : 0;
        __syncthreads();
        cnt_s[t] += v;
        __syncthreads();
    }
    int pos = cnt_s[t] - c;
    for (int i = lo; i < hi; ++i)
        if (flag[i]) list[pos++] = i;
    if (t == 1023) *count = cnt_s[1023];
    if (t == 0) {
        int m = 0x7fffffff;
        for (int w = 0; w < 32; ++w) m = min(m, first_s[w]);
        *first_unset = m == 0x7fffffff ? -1 : m;
    }
}

__global__ void k_keep_flags(Geometry g, const RangeInfo *ri, const DomainInfo *di, int dense, int *rkeep, int *dkeep)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < g.R) rkeep[i] = dense || !ri[i].shadow;
    if (i < g.D) {
        const DomainInfo d = di[i];
        dkeep[i] = dense || ((long long)g.m * d.Sqq - d.Sq * d.Sq) != 0;  // non-flat domain
    }
}

// Operand row j (j < count) of the range act[j]: centred pixels b - c_r.
__global__ void k_range_rows(Geometry g, const RangeInfo *ri, const uint16_t *bblk, const int *act, const int *nact,
                             float *rs32, __half *ra16)
{
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= *nact) return;
    const int r = act[j];
    const RangeInfo info = ri[r];
    for (int i = lane; i < g.m; i += 32) {
        const int bc = (int)bblk[(size_t)r * g.m + i] - info.c_r;
        if (rs32) rs32[(size_t)j * g.m + i] = (float)bc;
        if (ra16) {
            ra16[(size_t)j * g.KP + i] = __int2half_rn(bc);
            if (g.split_hilo) ra16[(size_t)j * g.KP + g.m + i] = __int2half_rn(bc);
        }
    }
    if (ra16) {
        const int base = g.split_hilo ? 2 * g.m : g.m;
        const int e_r = info.e_r;
        const int e_hi = (e_r >= 0) ? (e_r >> 10) : -((-e_r + 1023) >> 10);
        const int e_lo = e_r - 1024 * e_hi;
        for (int c = base + lane; c < g.KP; c += 32) {
            const int v = c == base ? e_hi : (c == base + 1 ? e_lo : 0);
            ra16[(size_t)j * g.KP + c] = __int2half_rn(v);
        }
    }
}

// Candidate rows 8j+k of the domain dact[j] (j < count): output pixel (y,x) of
// S_k(tau(d)) reads q at sym_src; domain constants in the same order.
__global__ void k_domain_rows(Geometry g, const DomainInfo *di, const uint16_t *qblk, const float4 *dconst,
                              const int *dact, const int *ndact, float *cb32, __half *cb16, float4 *dconst_c,
                              int *dmap)
{
    const int j = blockIdx.x;
    if (j >= *ndact) return;
    const int d = dact[j];
    const int i = threadIdx.x;  // blockDim = m
    const int n = g.n, m = g.m;
    const DomainInfo info = di[d];
    const int c_d = info.c_d, fd = info.f_d;
    if (i == 0) {
        dconst_c[j] = dconst[d];
        dmap[j] = d;
    }
    const int y = i >> g.ln, x = i & (n - 1);
    for (int k = 0; k < 8; ++k) {
        int sy, sx;
        sym_src(k, n, y, x, sy, sx);
        const int qc = (int)qblk[(size_t)d * m + (sy << g.ln) + sx] - c_d;
        const size_t row = (size_t)j * 8 + k;
        if (cb32) cb32[row * m + i] = (float)qc;
        if (cb16) {
            __half *rowp = cb16 + row * g.KP;
            if (g.split_hilo) {
                const int hi = (qc + 64) >> 7;  // floor; |hi| <= 128
                const int lo = qc - 128 * hi;   // in [-64, 63]
                rowp[i] = __int2half_rn(128 * hi);
                rowp[m + i] = __int2half_rn(lo);
            } else {
                rowp[i] = __int2half_rn(qc);
            }
            const int base = g.split_hilo ? 2 * m : m;
            if (i < g.KP - base) {
                float v = 0.0f;
                if (i == 0) v = -1024.0f * (float)fd / (float)m;
                if (i == 1) v = -(float)fd / (float)m;
                rowp[base + i] = __float2half_rn(v);
            }
        }
    }
}

cudaError_t launch_prep(const Geometry &g, const void *img, const EpiConst &ec, int dense, RangeInfo *ri,
                        DomainInfo *di, float4 *dconst, uint16_t *bblk, uint16_t *qblk, float *rs32, float *cb32,
                        __half *ra16, __half *cb16, int *tbest, const CompactBufs &cb, cudaStream_t st)
{
    k_range_prep<<<(g.R + 7) / 8, 256, 0, st>>>(g, ec, img, ri, bblk, tbest);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_domain_prep<<<g.D, g.m < 32 ? 32 : g.m, 0, st>>>(g, img, di, dconst, qblk);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int nmax = g.R > g.D ? g.R : g.D;
    k_keep_flags<<<(nmax + 255) / 256, 256, 0, st>>>(g, ri, di, dense, cb.rkeep, cb.dkeep);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_compact<<<1, 1024, 0, st>>>(g.R, cb.rkeep, cb.act, cb.counts + 0, cb.counts + 1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_compact<<<1, 1024, 0, st>>>(g.D, cb.dkeep, cb.dact, cb.counts + 2, cb.counts + 3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_range_rows<<<(g.R + 7) / 8, 256, 0, st>>>(g, ri, bblk, cb.act, cb.counts + 0, rs32, ra16);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_domain_rows<<<g.D, g.m, 0, st>>>(g, di, qblk, dconst, cb.dact, cb.counts + 2, cb32, cb16, cb.dconst_c, cb.dmap);
    return cudaGetLastError();
}

// Seed of the per-range best key: before the search, every range scores 256
// candidates -- the 8 symmetries of the 5 x 5 domains around it and of 7
// domains spread over the image -- from their exact cross terms, with the
// same code decision and key as the search epilogue.  Only clean keys (code
// not next to a rounding boundary, offset not clamped) are published: each is
// within the screening allowance of a real candidate's residual, which is all
// the search's insertion window needs.
__global__ void k_seed(Geometry g, EpiConst ec, const RangeInfo *ri, const DomainInfo *di, const float4 *dconst,
                       const uint16_t *bblk, const uint16_t *qblk, int *tbest)
{
    __shared__ unsigned b_s[kMaxM];
    __shared__ uint16_t q_s[kMaxM][32];  // [pixel][domain slot]: lanes read consecutive slots
    __shared__ int d_s[32];
    const int r = blockIdx.x;
    const RangeInfo rin = ri[r];  // block-uniform
    if (rin.shadow) return;
    if (threadIdx.x < 32) {
        const int slot_d = threadIdx.x;
        int d;
        if (slot_d < 25) {
            const int ry = (r / g.nx) * g.n, rx = (r % g.nx) * g.n;
            const int v0 = min(max((ry - g.n / 2) / g.t, 0), g.V - 1);
            const int u0 = min(max((rx - g.n / 2) / g.t, 0), g.U - 1);
            const int v = min(max(v0 + slot_d / 5 - 2, 0), g.V - 1);
            const int u = min(max(u0 + slot_d % 5 - 2, 0), g.U - 1);
            d = v * g.U + u;
        } else {
            d = (int)(((long long)r * 2654435761LL + (long long)(slot_d - 25) * 40503LL) % g.D);
        }
        d_s[slot_d] = d;
    }
    for (int i = threadIdx.x; i < g.m; i += blockDim.x) b_s[i] = bblk[(size_t)r * g.m + i];
    __syncthreads();
    const int lm = 2 * g.ln;  // log2(m)
    for (int e = threadIdx.x; e < 32 * g.m; e += blockDim.x) {
        const int sl = e >> lm, i = e & (g.m - 1);
        q_s[i][sl] = qblk[(size_t)d_s[sl] * g.m + i];
    }
    __syncthreads();
    const int k = threadIdx.x >> 5;     // one symmetry per warp: no divergence in sym_src
    const int slot_d = threadIdx.x & 31;
    const int d = d_s[slot_d];
    unsigned long long X = 0;
    for (int i = 0; i < g.m; ++i) {
        int sy, sx;
        sym_src(k, g.n, i >> g.ln, i & (g.n - 1), sy, sx);
        X += (unsigned)q_s[(sy << g.ln) + sx][slot_d] * b_s[i];
    }
    const DomainInfo dd = di[d];
    const long long num = (long long)g.m * (long long)X - dd.Sq * rin.Sb;  // exact
    const float Xt = __ll2float_rn(num) * ec.invm;
    const float4 c4 = dconst[d];
    const RangeEpi re = range_epi(rin, ec);
    float rho;
    const float c = epi_code(Xt, c4.x, ec, rho);
    if (fabsf(rho) > re.rho_lim) return;
    const float ostar = (re.Sb - c * c4.w * ec.inv4ls) * ec.invm;
    if (!(ostar < ec.pmax)) return;
    atomicMin(tbest + r, f2ord(epi_key(Xt, c, re.zb, c4, ec)));
}

cudaError_t launch_seed(const Geometry &g, const EpiConst &ec, const RangeInfo *ri, const DomainInfo *di,
                        const float4 *dconst, const uint16_t *bblk, const uint16_t *qblk, int *tbest,
                        cudaStream_t st)
{
    k_seed<<<g.R, 256, 0, st>>>(g, ec, ri, di, dconst, bblk, qblk, tbest);
    return cudaGetLastError();
}

}  // namespace fic
