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

// Lanes per range or domain in the statistics kernel: G = m / 8 (8 pixels a
// lane; m = 256 takes the whole warp), so a warp holds 32 / G items whose
// sums reduce within their lane groups and whose per-item tails run side by
// side.
__host__ __device__ constexpr int stats_group(int m) { return m >= 256 ? 32 : m / 8; }
__host__ __device__ constexpr int stats_items(int m) { return 8 * (32 / stats_group(m)); }  // per block
__host__ __device__ __forceinline__ int stats_range_blocks(const Geometry &g)
{
    return (g.R + stats_items(g.m) - 1) / stats_items(g.m);
}
__host__ __device__ __forceinline__ int stats_blocks(const Geometry &g)
{
    return stats_range_blocks(g) + (g.D + stats_items(g.m) - 1) / stats_items(g.m);
}

// Sum over the G lanes of a group (G a power of two; every lane of the warp
// takes part).
template <typename T>
__device__ __forceinline__ T group_sum(T v, int G)
{
    for (int off = G >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// G lanes per range (li = lane within the group, 8 pixels each): statistics,
// centre, allowances, and the keep flag (every range but shadow ranges, or
// all when dense).  `valid` is false for the lanes of a group past the last
// range: they take part in the reductions only.
template <int LN, bool B8>
__device__ __forceinline__ bool range_stats(const Geometry &g, const EpiConst &ec, const void *img, int dense,
                                            int tc_mode, const int *active, int r, bool valid, int li, int G,
                                            RangeInfo *ri, uint16_t *bblk, int *tbest, int *rkeep)
{
    constexpr int n = 1 << LN, m = n * n;
    const int rr = valid ? r : 0;
    const int ry = (rr / g.nx) * n, rx = (rr % g.nx) * n;
    int bv[8];
    long long Sb = 0, Sbb = 0;
    int bmin = 1 << 30, bmax = -1;
    // every load issued before the first use (no store between them)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int i = li + G * j;
        const size_t off = (size_t)(ry + (i >> LN)) * g.pitch + rx + (i & (n - 1));
        bv[j] = valid ? (B8 ? (int)((const uint8_t *)img)[off] : (int)((const uint16_t *)img)[off]) : 0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int b = bv[j];
        Sb += b;
        Sbb += (long long)b * b;
        bmin = min(bmin, b);
        bmax = max(bmax, b);
        if (valid) bblk[(size_t)rr * m + li + G * j] = (uint16_t)b;
    }
    Sb = group_sum(Sb, G);
    Sbb = group_sum(Sbb, G);
    for (int off = G >> 1; off > 0; off >>= 1) {
        bmin = min(bmin, __shfl_xor_sync(0xffffffffu, bmin, off));
        bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, off));
    }
    if (!valid || li != 0) return false;
    // centre: nearest integer to the mean, kept within 2048 of every pixel so
    // that b - c_r is an exact FP16 integer
    long long cr = (2 * Sb + m) >> (2 * LN + 1);  // m = 2^(2 ln), Sb >= 0
    cr = max((long long)(bmax - 2048), min((long long)(bmin + 2048), cr));
    const int c_r = (int)cr;
    const int e_r = (int)(Sb - (long long)m * c_r);
    // sum (b - c_r)^2, exactly
    const float bp2f = __ll2float_rn(Sbb - 2 * cr * Sb + (long long)m * cr * cr);
    // per-range constants: integer arithmetic and FP32 only (the FP64 rate of
    // this part is a small fraction of FP32)
    RangeInfo info;
    info.Sb = Sb;
    info.Sbb = Sbb;
    info.c_r = c_r;
    info.e_r = e_r;
    constexpr float invm = 1.0f / (float)m;
    info.sbbc = (float)((long long)m * Sbb - Sb * Sb) * invm;
    const int z = 4 * g.Ls * (int)Sb;  // < 2^31 for B <= 12, m <= 256, s_bits <= 8
    info.zb = (float)(g.mod_g ? z % g.Gi : z);
    info.bp2 = bp2f;
    // FP32 error of Ls*s: ~1e-6 when the cross term is exact, plus the
    // accumulation error of high-variance pairs (grows with sum (b-c_r)^2):
    // FP32 sums of integer products are exact below 2^24, so an error needs
    // |q'| |b'| above it, and is then at most K u |q'| |b'|, which moves Ls*s
    // by at most ~4 Ls K u^2 |b'|^2 (den ~ m |q'|^2), u = 2^-24, K = m terms.
    // tc_mode 1 (the tensor-core search's separate hi/lo accumulators, K <=
    // 64): the cross term X' is exact but for the rounding of hi + lo and of
    // the folded correction: relative errors of 2^-23 of (|X'| + |corr|),
    // |corr| <= |e_r|/2, times alpha <= 2m/(m-1) < 2.1 and 2 Ls.  tc_mode 2
    // (tensor cores with K = 256 per part): both error sources, the
    // accumulation bound doubled (the hardware's order of the FP32 additions
    // is not specified).
    const float er_abs = fabsf((float)e_r);
    const float acc_err = 12.0f * g.Ls * (float)(m > 64 ? m : 64) * bp2f * 3.552713678800501e-15f;  // 2^-48
    const float eta = tc_mode == 1   ? 1e-5f + 1.2e-7f * g.Ls * (2.0f + 2.1f * er_abs)
                      : tc_mode == 2 ? 1e-5f + 2.0f * acc_err + 1.2e-7f * g.Ls * (2.0f + 2.1f * er_abs)
                                     : 1e-5f + acc_err;
    info.rho_lim = 0.5f - fminf(eta, 0.25f);
    // Screening allowance.  A candidate within reach of the winner has
    // |c| * sqrt(sum (q-q_mean)^2) <= 4*Ls*(sqrt(Sbb_c) + sqrt(R)), R <= Eb; its
    // centred products (hi/lo split included) then sum to at most S.  Below
    // 2^23 every FP32 partial sum of integers is exact and the cross term
    // carries no error; otherwise allow 2^-15 relative.
    const float sbbc = fmaxf(info.sbbc, 0.0f);
    const float Eb = 4.0f * (sbbc + ec.delta_o);
    const float sb = sqrtf(bp2f);
    const float sqm = n;  // sqrt(m)
    const float S = (4.0f * g.Ls * (sqrtf(sbbc) + sqrtf(Eb)) + sqm) * sb + (g.split_hilo ? 128.0f * sqm * sb : 0.0f);
    const bool exact = tc_mode == 1 || S < 8.0e6f;  // < 2^23 with margin, or exact partial sums
    const float gam = 3.0517578125e-05f;  // 2^-15
    const float corr_a = tc_mode != 0 ? 9.5367431640625e-07f * g.Ls * er_abs : 0.0f;  // 2^-20: the folded correction
    info.beta_q = exact ? 0.0f : 4.0f * g.Ls * gam * sb;
    info.beta_a = 3.814697265625e-06f * 2.0f * g.Ls * (sbbc + ec.delta_o) + 1e-3f + corr_a +
                  (exact ? 0.0f : gam * g.Ls * 128.0f * sqm * sb);
    info.shadow = bmin == bmax ? 1 : 0;
    info.pad = 0;
    ri[r] = info;
    tbest[r] = 0x7f800000;  // +inf in the ordered-integer encoding of floats
    const bool keep = (!active || active[r]) && (dense || !info.shadow);
    rkeep[r] = keep;
    return keep;
}


// G lanes per domain (li = lane within the group, 8 contracted pixels
// each): the 2x2 sums q (tau as an integer sum, the mean being q/4), Sq, Sqq,
// centre, the epilogue column constants, and the keep flag (every domain but
// flat ones, den = 0, or all when dense).
template <int LN, bool B8>
__device__ __forceinline__ bool domain_stats(const Geometry &g, const void *img, int dense, int d, bool valid,
                                             int li, int G, DomainInfo *di, float4 *dconst, uint16_t *qblk,
                                             int *dkeep)
{
    constexpr int n = 1 << LN, m = n * n;
    const int dd0 = valid ? d : 0;
    const int dy = (dd0 / g.U) * g.t, dx = (dd0 % g.U) * g.t;
    long long Sq = 0, Sqq = 0;
    int qv[8];
    // every load issued before the first store
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int i = li + G * j;
        const int y = i >> LN, x = i & (n - 1);
        const size_t o0 = (size_t)(dy + 2 * y) * g.pitch + dx + 2 * x;
        int q = 0;
        if (valid) {
            if (B8) {
                const uint8_t *p8 = (const uint8_t *)img;
                q = (int)p8[o0] + (int)p8[o0 + 1] + (int)p8[o0 + g.pitch] + (int)p8[o0 + g.pitch + 1];
            } else {
                const uint16_t *p16 = (const uint16_t *)img;
                q = (int)p16[o0] + (int)p16[o0 + 1] + (int)p16[o0 + g.pitch] + (int)p16[o0 + g.pitch + 1];
            }
        }
        qv[j] = q;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int q = qv[j];
        if (valid) qblk[(size_t)d * m + li + G * j] = (uint16_t)q;
        Sq += q;
        Sqq += (long long)q * q;
    }
    Sq = group_sum(Sq, G);
    Sqq = group_sum(Sqq, G);
    if (!valid || li != 0) return false;
    const long long cd = (2 * Sq + m) >> (2 * LN + 1);  // m = 2^(2 ln), Sq >= 0
    const long long den = (long long)m * Sqq - Sq * Sq;
    DomainInfo info;
    info.Sq = Sq;
    info.Sqq = Sqq;
    info.c_d = (int)cd;
    info.f_d = (int)(Sq - (long long)m * cd);
    info.qp2 = 0.0f;
    info.pad = 0.0f;
    di[d] = info;
    // FP32 from exact integers (no FP64 on this path)
    float4 c4;
    const float denf = (float)den;
    c4.x = den > 0 ? (2.0f * m) / denf : 0.0f;
    c4.y = (float)(g.mod_g ? (int)Sq % g.Gi : (int)Sq);
    c4.z = denf / (8.0f * m * g.Ls);
    c4.w = (float)Sq;
    dconst[d] = c4;
    const bool keep = dense || den != 0;
    dkeep[d] = keep;
    return keep;
}

// Statistics of every range (the first stats_range_blocks blocks) and every
// domain (the blocks after), one launch; stats_items per block of 256.
template <int LN, bool B8>
__device__ __forceinline__ void stats_block(const Geometry &g, const EpiConst &ec, const void *img, int dense,
                                            int tc_mode, const int *active, RangeInfo *ri, uint16_t *bblk,
                                            int *tbest, DomainInfo *di, float4 *dconst, uint16_t *qblk, int *rkeep,
                                            int *dkeep, int *zero4, uint4 *bmask, int *bcount, int bx)
{
    if (bx == 0 && threadIdx.x < 4) zero4[threadIdx.x] = 0;  // exact-scan queue counters
    constexpr int G = stats_group(1 << (2 * LN)), per_block = stats_items(1 << (2 * LN));
    static_assert(per_block <= 128, "the keep mask of a block is four words");
    const int rbs = stats_range_blocks(g);
    const int li = threadIdx.x & (G - 1);
    const int item = threadIdx.x / G;  // (warp, group) in order
    bool keep;
    if (bx < rbs) {
        const int r = bx * per_block + item;
        keep = range_stats<LN, B8>(g, ec, img, dense, tc_mode, active, r, r < g.R, li, G, ri, bblk, tbest, rkeep);
    } else {
        const int d = (bx - rbs) * per_block + item;
        keep = domain_stats<LN, B8>(g, img, dense, d, d < g.D, li, G, di, dconst, qblk, dkeep);
    }
    if (!bmask) return;
    // the block's keep flags in item order (bit i of word i / 32) and their
    // count, for the compaction that follows without a scan launch
    __shared__ int keep_s[per_block];
    if (li == 0) keep_s[item] = keep ? 1 : 0;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t w[4];
        int total = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int it = 32 * k + threadIdx.x;
            w[k] = __ballot_sync(0xffffffffu, it < per_block && keep_s[it] != 0);
            total += __popc(w[k]);
        }
        if (threadIdx.x == 0) {
            bmask[bx] = make_uint4(w[0], w[1], w[2], w[3]);
            bcount[bx] = total;
        }
    }
}

template <int LN, bool B8>
__global__ void __launch_bounds__(256) k_stats(Geometry g, EpiConst ec, const void *img, int dense, int tc_mode,
                                               const int *active, RangeInfo *ri, uint16_t *bblk, int *tbest,
                                               DomainInfo *di, float4 *dconst, uint16_t *qblk, int *rkeep,
                                               int *dkeep, int *zero4, uint4 *bmask, int *bcount)
{
    grid_dep_sync();
    stats_block<LN, B8>(g, ec, img, dense, tc_mode, active, ri, bblk, tbest, di, dconst, qblk, rkeep, dkeep, zero4,
                        bmask, bcount, blockIdx.x);
}

// Batched: blockIdx.y = slice.
template <int LN, bool B8>
__global__ void __launch_bounds__(256) k_stats_batch(const SliceCtx *__restrict__ ctx, int dense, int tc_mode)
{
    grid_dep_sync();
    const SliceCtx c = ctx[blockIdx.y];
    if ((int)blockIdx.x >= stats_blocks(c.g)) return;
    const EncBufs &b = c.b;
    stats_block<LN, B8>(c.g, c.ec, c.img, dense, tc_mode, nullptr, b.ri, b.bblk, b.tbest, b.di, b.dconst, b.qblk,
                        b.cb.rkeep, b.cb.dkeep, b.fb_count, nullptr, nullptr, blockIdx.x);
}

// The statistics kernels of a geometry (range size and 8-bit pixels are
// template parameters): calls launch(single, batched).
template <typename Launch>
static cudaError_t with_stats_kernel(const Geometry &g, Launch &&launch)
{
    const bool b8 = g.B <= 8;
    switch (g.ln) {
    case 2: return b8 ? launch(k_stats<2, true>, k_stats_batch<2, true>) : launch(k_stats<2, false>, k_stats_batch<2, false>);
    case 3: return b8 ? launch(k_stats<3, true>, k_stats_batch<3, true>) : launch(k_stats<3, false>, k_stats_batch<3, false>);
    case 4: return b8 ? launch(k_stats<4, true>, k_stats_batch<4, true>) : launch(k_stats<4, false>, k_stats_batch<4, false>);
    default: return cudaErrorInvalidValue;
    }
}

// Stable compaction of the flagged items by one block of T threads, over
// the ranges or over the domains: the kept indices in their original order,
// cnt[0] = how many, cnt[1] = the first unflagged index (-1 if none).
// Passes of 16 x T items: every flag of a pass is loaded up front (one
// memory latency), warp ballots give per-(round, warp) counts, one warp scans
// those counts in item order, and every thread scatters its kept items.
constexpr int kCompactRounds = 16;
template <int T>
__device__ __forceinline__ void compact_block(int nr, const int *rflag, int *ract, int *rcnt, int nd,
                                              const int *dflag, int *dact, int *dcnt, bool dom)
{
    constexpr int W = T / 32;             // warps
    constexpr int E = kCompactRounds * W / 32;  // counts per lane of the scanning warp
    static_assert(T % 64 == 0 && T <= 1024, "two or more warps, at most 1024 threads");
    __shared__ int off_s[kCompactRounds * W];
    __shared__ int base_s, first_s;
    const int n = dom ? nd : nr;
    const int *flag = dom ? dflag : rflag;
    int *list = dom ? dact : ract;
    int *cnt = dom ? dcnt : rcnt;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) {
        base_s = 0;
        first_s = 0x7fffffff;
    }
    int fu = 0x7fffffff;
    for (int c0 = 0; c0 < n; c0 += T * kCompactRounds) {
        // all the pass's flag loads in flight at once (clamped index: no
        // branch between them)
        int fv[kCompactRounds];
#pragma unroll
        for (int q = 0; q < kCompactRounds; ++q) fv[q] = flag[min(c0 + q * T + t, n - 1)];
        bool f[kCompactRounds];
#pragma unroll
        for (int q = 0; q < kCompactRounds; ++q) {
            const int i = c0 + q * T + t;
            f[q] = i < n && fv[q] != 0;
            if (i < n && !f[q]) fu = min(fu, i);
        }
        unsigned b[kCompactRounds];
#pragma unroll
        for (int q = 0; q < kCompactRounds; ++q) {
            b[q] = __ballot_sync(0xffffffffu, f[q]);
            if (lane == 0) off_s[q * W + w] = __popc(b[q]);
        }
        __syncthreads();
        if (w == 0) {
            // exclusive scan of the 16 W counts in item order; lane l owns
            // entries [E l, E l + E)
            int v[E], sum = 0;
#pragma unroll
            for (int q = 0; q < E; ++q) {
                v[q] = off_s[E * lane + q];
                sum += v[q];
            }
            int x = sum;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            const int base = base_s;
            int run = base + x - sum;
#pragma unroll
            for (int q = 0; q < E; ++q) {
                off_s[E * lane + q] = run;
                run += v[q];
            }
            __syncwarp();
            if (lane == 31) base_s = base + x;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kCompactRounds; ++q)
            if (f[q]) list[off_s[q * W + w] + __popc(b[q] & ((1u << lane) - 1u))] = c0 + q * T + t;
        __syncthreads();  // off_s is rewritten by the next pass
    }
    for (int o = 16; o > 0; o >>= 1) fu = min(fu, __shfl_xor_sync(0xffffffffu, fu, o));
    if (lane == 0) atomicMin(&first_s, fu);
    __syncthreads();
    if (t == 0) {
        cnt[0] = base_s;
        cnt[1] = first_s == 0x7fffffff ? -1 : first_s;
    }
}


// FP16 bit pattern of an integer of magnitude below 2^11 (exact).
__device__ __forceinline__ uint32_t h16(int v) { return __half_as_ushort(__int2half_rn(v)); }

// Reverses the order of the 8 (4) FP16 values of v when sel = 0x5476 (sel =
// 0x3210 leaves them): each output word takes the mirrored input word with
// its halves swapped.
__device__ __forceinline__ uint4 rev8_sel(uint4 v, uint32_t sel)
{
    return make_uint4(__byte_perm(v.x, v.w, sel), __byte_perm(v.y, v.z, sel), __byte_perm(v.z, v.y, sel),
                      __byte_perm(v.w, v.x, sel));
}

__device__ __forceinline__ uint2 rev4_sel(uint2 v, uint32_t sel)
{
    return make_uint2(__byte_perm(v.x, v.y, sel), __byte_perm(v.y, v.x, sel));
}

// Operand row shapes for ranges of 2^LN x 2^LN pixels; SPLIT: q' is split
// into hi/lo FP16 parts (bit depths above 8).
template <int LN, bool SPLIT>
struct RowShape {
    static constexpr int n = 1 << LN, m = n * n;
    static constexpr int base = SPLIT ? 2 * m : m;  // first column after the pixel parts
    static constexpr int KP = base + 16;             // FP16 row length (Geometry::KP)
    static constexpr int nch = KP / 8;               // 16-byte chunks per row
};

// Operand row j (j < count) of the range r: centred pixels b - c_r (twice
// when q is split into hi/lo parts), then e_hi, e_lo (e_r = 1024 e_hi + e_lo)
// and zeros.  FP16 layout: one 16-byte chunk per lane, 8 pixels converted
// from one 16-byte load of the range's pixels.
template <int LN, bool SPLIT>
__device__ __forceinline__ void range_row(const RangeInfo *ri, const uint16_t *bblk, int j, int r, int lane,
                                          float *rs32, __half *ra16)
{
    typedef RowShape<LN, SPLIT> S;
    const int c_r = ri[r].c_r;
    if (ra16) {
        const int e_r = ri[r].e_r;
        const int e_hi = (e_r >= 0) ? (e_r >> 10) : -((-e_r + 1023) >> 10);
        const int e_lo = e_r - 1024 * e_hi;
        uint4 *row = reinterpret_cast<uint4 *>(ra16 + (size_t)j * S::KP);
        const uint4 *src = reinterpret_cast<const uint4 *>(bblk + (size_t)r * S::m);
        for (int c = lane; c < S::nch; c += 32) {
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (c < S::base / 8) {
                const uint4 w = src[SPLIT && c >= S::m / 8 ? c - S::m / 8 : c];
                v.x = h16((int)(w.x & 0xffffu) - c_r) | (h16((int)(w.x >> 16) - c_r) << 16);
                v.y = h16((int)(w.y & 0xffffu) - c_r) | (h16((int)(w.y >> 16) - c_r) << 16);
                v.z = h16((int)(w.z & 0xffffu) - c_r) | (h16((int)(w.z >> 16) - c_r) << 16);
                v.w = h16((int)(w.w & 0xffffu) - c_r) | (h16((int)(w.w >> 16) - c_r) << 16);
            } else if (c == S::base / 8) {
                v.x = h16(e_hi) | (h16(e_lo) << 16);
            }
            row[c] = v;
        }
    }
    if (rs32) {
        for (int i = lane; i < S::m; i += 32) rs32[(size_t)j * S::m + i] = (float)((int)bblk[(size_t)r * S::m + i] - c_r);
    }
}

// Per-lane constants of the FP16 domain rows: lane = 4 k + c0 writes chunks
// c0, c0 + 4, ... of the row of symmetry k, whose flags are fixed per lane.
struct RowLane {
    int k;
    int part;      // staging part read: + 2 m when S_k swaps the axes (transposed copies)
    int rm, cm;    // row and column masks in the part read
    uint32_t sel;  // byte selector: reverse the chunk when the column mask is set
};

template <int LN>
__device__ __forceinline__ RowLane row_lane(int lane)
{
    constexpr int n = 1 << LN, m = n * n;
    const SymFlags f = sym_flags(lane >> 2, n);
    RowLane L;
    L.k = lane >> 2;
    L.part = f.swap ? 2 * m : 0;
    L.rm = f.swap ? f.mx : f.my;
    L.cm = f.swap ? f.my : f.mx;
    L.sel = L.cm ? 0x5476u : 0x3210u;
    return L;
}

// Candidate rows 8j+k of the domain d: output pixel i = (y,x) of
// S_k(tau(d)) is q at sym_src_index(k, i), centred by c_d.  FP16 row
// (tensor-core layout): [128*hi | lo (12-bit only) | -1024 f_d/m, -f_d/m,
// 0...] with q - c_d = 128*hi + lo.  The warp converts the domain's m values
// once into FP16 bit patterns in shared memory (st: hi, lo, then both
// transposed), then writes the 16-byte chunks of the 8 rows: under S_k the 8
// values of a chunk are a run along one row of a staged part (of the
// transposed part when S_k swaps the axes), reversed when S_k flips the
// columns (n >= 8: one run of 8; n = 4: two runs of 4).  SIMT layout (cb32):
// the 8 symmetric copies of q - c_d in FP32.  Domain constants in the same
// order.
template <int LN, bool SPLIT>
__device__ __forceinline__ void domain_rows_warp(const DomainInfo *di, const uint16_t *qblk, const float4 *dconst, int j,
                                                 int d, int lane, const RowLane &rl, uint16_t *st, float *cb32,
                                                 __half *cb16, float4 *dconst_c, int *dmap)
{
    typedef RowShape<LN, SPLIT> S;
    constexpr int n = S::n, m = S::m;
    constexpr int QPL = (m + 31) / 32;
    int qv[QPL];
#pragma unroll
    for (int u = 0; u < QPL; ++u) {  // every load before the first store
        const int i = lane + 32 * u;
        qv[u] = i < m ? (int)qblk[(size_t)d * m + i] : 0;
    }
    const int c_d = di[d].c_d, fd = di[d].f_d;
    if (lane == 0) {
        dconst_c[j] = dconst[d];
        dmap[j] = d;
    }
#pragma unroll
    for (int u = 0; u < QPL; ++u) {
        const int i = lane + 32 * u;
        if (i < m) {
            const int qc = qv[u] - c_d;
            const int it = ((i & (n - 1)) << LN) + (i >> LN);  // transposed position
            if (cb32) {
                st[i] = (uint16_t)(qc + 32768);  // SIMT operand: centred value, biased
            } else if (SPLIT) {
                const int hi = (qc + 64) >> 7;  // floor; |hi| <= 128
                const uint16_t h = (uint16_t)h16(128 * hi), l = (uint16_t)h16(qc - 128 * hi);
                st[i] = h;
                st[m + i] = l;
                st[2 * m + it] = h;
                st[3 * m + it] = l;
            } else {
                const uint16_t h = (uint16_t)h16(qc);
                st[i] = h;
                st[2 * m + it] = h;
            }
        }
    }
    __syncwarp();
    if (cb32) {
        for (int k = 0; k < 8; ++k) {
            const SymFlags f = sym_flags(k, n);
            for (int i = lane; i < m; i += 32)
                cb32[((size_t)j * 8 + k) * m + i] =
                    (float)((int)st[sym_src_index(f, LN, i >> LN, i & (n - 1))] - 32768);
        }
        return;
    }
    // tail: -f_d/m in the scale of the hi part and of the lo part (m is a
    // power of two: the products are the exact quotients)
    const uint32_t tail = (uint32_t)__half_as_ushort(__float2half_rn((float)fd * (-1024.0f / m))) |
                          ((uint32_t)__half_as_ushort(__float2half_rn((float)fd * (-1.0f / m))) << 16);
    uint4 *row = reinterpret_cast<uint4 *>(cb16 + ((size_t)j * 8 + rl.k) * S::KP);
    constexpr int NI = (S::nch + 3) / 4;
#pragma unroll
    for (int it = 0; it < NI; ++it) {
        const int c = (lane & 3) + 4 * it;
        if (c >= S::nch) break;
        const int col0 = 8 * c;
        uint4 v;
        if (col0 >= S::base) {
            v = make_uint4(col0 == S::base ? tail : 0u, 0u, 0u, 0u);
        } else {
            const bool lo_part = SPLIT && col0 >= m;  // second copy (12-bit only)
            const int i0 = lo_part ? col0 - m : col0;
            const uint16_t *b = st + rl.part + (lo_part ? m : 0);
            if (n >= 8) {
                const int y = i0 >> LN, x0 = i0 & (n - 1);
                v = rev8_sel(*reinterpret_cast<const uint4 *>(b + ((y ^ rl.rm) << LN) + ((x0 ^ rl.cm) & ~7)), rl.sel);
            } else {
                const int y = i0 >> 2;
                const uint2 r0 = rev4_sel(*reinterpret_cast<const uint2 *>(b + ((y ^ rl.rm) << 2)), rl.sel);
                const uint2 r1 = rev4_sel(*reinterpret_cast<const uint2 *>(b + (((y + 1) ^ rl.rm) << 2)), rl.sel);
                v = make_uint4(r0.x, r0.y, r1.x, r1.y);
            }
        }
        row[c] = v;
    }
}

// Operand rows of the kept ranges (a warp per row) and of the kept domains
// (a warp per domain), one launch.  The rows come in groups of 8 (one per
// warp): first the range groups, then the domain groups, as many as the
// compaction kept; block `first` takes every stride-th group, so a grid of
// resident blocks covers them with no block spent on nothing.
// Resident blocks per SM: 5 at 48 registers x 256 threads; 4 (64 registers)
// for 16x16 ranges, whose 8 pixels a lane would not fit in 48 without spills.
__host__ __device__ constexpr int rows_blocks_per_sm(int ln) { return ln == 4 ? 4 : 5; }
template <int LN, bool SPLIT>
__device__ __forceinline__ void rows_block(const RangeInfo *ri, const uint16_t *bblk, const DomainInfo *di,
                                           const uint16_t *qblk, const float4 *dconst, const int *act,
                                           const int *dact, const int *counts, float *rs32, __half *ra16,
                                           float *cb32, __half *cb16, float4 *dconst_c, int *dmap, int first,
                                           int stride)
{
    constexpr int m = 1 << (2 * LN);
    __shared__ __align__(16) uint16_t st_s[8][4 * m];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const RowLane rl = row_lane<LN>(lane);
    const int nr = counts[0], nd = counts[2];
    const int rgroups = (nr + 7) / 8, groups = rgroups + (nd + 7) / 8;
    for (int vb = first; vb < groups; vb += stride) {
        if (vb < rgroups) {
            const int j = vb * 8 + w;
            if (j < nr) range_row<LN, SPLIT>(ri, bblk, j, act[j], lane, rs32, ra16);
        } else {
            const int j = (vb - rgroups) * 8 + w;
            if (j < nd) {
                __syncwarp();  // the warp's staging area of its previous domain is read
                domain_rows_warp<LN, SPLIT>(di, qblk, dconst, j, dact[j], lane, rl, st_s[w], cb32, cb16, dconst_c,
                                            dmap);
            }
        }
    }
}

template <int LN, bool SPLIT>
__global__ void __launch_bounds__(256, rows_blocks_per_sm(LN)) k_rows(const RangeInfo *ri, const uint16_t *bblk,
                                              const DomainInfo *di, const uint16_t *qblk, const float4 *dconst,
                                              const int *act, const int *dact, const int *counts, float *rs32,
                                              __half *ra16, float *cb32, __half *cb16, float4 *dconst_c, int *dmap)
{
    grid_dep_sync();
    rows_block<LN, SPLIT>(ri, bblk, di, qblk, dconst, act, dact, counts, rs32, ra16, cb32, cb16, dconst_c, dmap,
                          blockIdx.x, gridDim.x);
}

template <int LN, bool SPLIT>
__global__ void __launch_bounds__(256, rows_blocks_per_sm(LN)) k_rows_batch(const SliceCtx *__restrict__ ctx)
{
    grid_dep_sync();
    const SliceCtx &c = ctx[blockIdx.y];
    const EncBufs &b = c.b;
    rows_block<LN, SPLIT>(b.ri, b.bblk, b.di, b.qblk, b.dconst, b.cb.act, b.cb.dact, b.cb.counts, b.rs32, b.ra16,
                          b.cb32, b.cb16, b.cb.dconst_c, b.cb.dmap, blockIdx.x, gridDim.x);
}

// The row kernels of a geometry (range size and hi/lo split are template
// parameters): calls launch(single, batched).
template <typename Launch>
static cudaError_t with_rows_kernel(const Geometry &g, Launch &&launch)
{
    const bool sp = g.split_hilo != 0;
    switch (g.ln) {
    case 2: return sp ? launch(k_rows<2, true>, k_rows_batch<2, true>) : launch(k_rows<2, false>, k_rows_batch<2, false>);
    case 3: return sp ? launch(k_rows<3, true>, k_rows_batch<3, true>) : launch(k_rows<3, false>, k_rows_batch<3, false>);
    case 4: return sp ? launch(k_rows<4, true>, k_rows_batch<4, true>) : launch(k_rows<4, false>, k_rows_batch<4, false>);
    default: return cudaErrorInvalidValue;
    }
}


// Seed of the per-range best key: before the search, every range scores the
// 8 symmetries of a few domains -- the ones around it and 7 spread over the
// image -- from their exact cross terms, with the same code decision and key
// as the search epilogue.  Only clean keys (code not next to a rounding
// boundary, offset not clamped) are published: each is within the screening
// allowance of a real candidate's residual, which is all the search's
// insertion window needs.
//
// seed_warp (m = 256): one warp per range over 32 domain slots (5 x 5 + 7),
// lane = slot, all 8 symmetries per lane: bk[k][j] is the range pixel that
// S_k places over domain pixel j, so X(d, k) = sum_j q_d[j] * bk[k][j];
// q2[p][slot] holds the contracted-domain pixels 2p, 2p+1 of the slot's
// domain (lanes read consecutive words, the bk reads are broadcasts); 8 m
// ints of bk and m/2 x 32 words of q2 per warp.  seed_range (m <= 64): the
// same over 16 slots (3 x 3 + 7), the warp's two halves taking four
// symmetries each.  The loads of a warp are issued together (one round trip
// after the keep flag).
__host__ __device__ constexpr int seed_warps(int m) { return m <= 64 ? 16 : 8; }
// Shared ints per seed warp: one range (m = 256: 8 m of bk, 16 m of q2;
// m <= 64, see seed_range: 8 (m + 4) of bk, 8 m of q2).
__host__ __device__ constexpr int seed_warp_ints(int m) { return m <= 64 ? 16 * m + 32 : 24 * m; }
__host__ __device__ constexpr size_t seed_smem(int m) { return sizeof(int) * (size_t)seed_warps(m) * seed_warp_ints(m); }

template <int PPL>  // range pixels per lane, at least m / 32
__device__ __forceinline__ void seed_warp(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                                          const DomainInfo *di, const float4 *dconst, const uint16_t *bblk,
                                          const uint16_t *qblk, const int *rkeep, int *tbest, int r, int lane,
                                          int *bk, uint32_t *q2)
{
    if (!rkeep[r]) return;  // warp-uniform: a range that is not screened
    int d;
    if (lane < 25) {
        const int ry = (r / g.nx) * g.n, rx = (r % g.nx) * g.n;
        const int v0 = min(max((ry - g.n / 2) / g.t, 0), g.V - 1);
        const int u0 = min(max((rx - g.n / 2) / g.t, 0), g.U - 1);
        const int v = min(max(v0 + lane / 5 - 2, 0), g.V - 1);
        const int u = min(max(u0 + lane % 5 - 2, 0), g.U - 1);
        d = v * g.U + u;
    } else {
        d = (int)(((long long)r * 2654435761LL + (long long)(lane - 25) * 40503LL) % g.D);
    }
    int bv[PPL];
#pragma unroll
    for (int j = 0; j < PPL; ++j) {
        const int i = lane + 32 * j;
        bv[j] = i < g.m ? (int)bblk[(size_t)r * g.m + i] : 0;
    }
    const uint4 *qrow = reinterpret_cast<const uint4 *>(qblk + (size_t)d * g.m);
    const int nv = g.m >> 3;  // 16-byte vectors of the slot's domain row
    uint4 qv[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) qv[v] = v < nv ? __ldg(qrow + v) : make_uint4(0, 0, 0, 0);
    const RangeInfo rin = ri[r];
    const DomainInfo dd = di[d];
    const float4 c4 = dconst[d];
#pragma unroll
    for (int j = 0; j < PPL; ++j) {
        const int i = lane + 32 * j;
        if (i < g.m) {
            const int y = i >> g.ln, x = i & (g.n - 1);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                int sy, sx;
                sym_src(k, g.n, y, x, sy, sx);
                bk[k * g.m + (sy << g.ln) + sx] = bv[j];
            }
        }
    }
    for (int v0 = 0; v0 < nv; v0 += 8) {
        if (v0 > 0) {  // rows longer than 8 vectors (m = 256)
#pragma unroll
            for (int v = 0; v < 8; ++v) qv[v] = v0 + v < nv ? __ldg(qrow + v0 + v) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            if (v0 + v < nv) {
                q2[(4 * (v0 + v) + 0) * 32 + lane] = qv[v].x;
                q2[(4 * (v0 + v) + 1) * 32 + lane] = qv[v].y;
                q2[(4 * (v0 + v) + 2) * 32 + lane] = qv[v].z;
                q2[(4 * (v0 + v) + 3) * 32 + lane] = qv[v].w;
            }
        }
    }
    __syncwarp();
    unsigned long long X[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) X[k] = 0;
    for (int p0 = 0; p0 < (g.m >> 1); p0 += 4) {
        // eight products of at most 4P * P < 2^26 per partial: exact in 32 bits
        uint32_t s8[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) s8[k] = 0;
#pragma unroll
        for (int p = p0; p < p0 + 4; ++p) {
            const uint32_t w = q2[p * 32 + lane];
            const uint32_t qa = w & 0xffffu, qb = w >> 16;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int2 b2 = *reinterpret_cast<const int2 *>(bk + k * g.m + 2 * p);
                s8[k] += qa * (uint32_t)b2.x + qb * (uint32_t)b2.y;
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) X[k] += s8[k];
    }
    const RangeEpi re = range_epi(rin, ec);
    const long long sqsb = dd.Sq * rin.Sb;
    int best = 0x7fffffff;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const long long num = (long long)g.m * (long long)X[k] - sqsb;  // exact
        const float Xt = __ll2float_rn(num) * ec.invm;
        float rho;
        const float c = epi_code(Xt, c4.x, 0.5f, ec, rho);
        if (fabsf(rho) > re.rho_lim) continue;
        const float ostar = (re.Sb - c * c4.w * ec.inv4ls) * ec.invm;
        if (!(ostar < ec.pmax)) continue;
        best = min(best, f2ord(epi_key(Xt, -0.0f, c, re.zb, c4, ec)));
    }
    best = __reduce_min_sync(0xffffffffu, best);
    if (lane == 0 && best != 0x7fffffff) atomicMin(tbest + r, best);
}

// The seed of one range (m <= 64) by a whole warp: the same scoring as
// seed_warp over 16 domain slots -- the 3 x 3 domains around the range and 7
// spread over the image -- with lane = (symmetry half h, slot sl): the lane
// scores symmetries 4h .. 4h+3 of its slot's domain.  bk holds the range's
// symmetry-permuted pixels (rows of m + 4 ints: 16-byte aligned, and the two
// halves' broadcast reads fall in different banks), q2[pp][slot] the slots'
// domain pixels 4 pp .. 4 pp + 3 as two words (each slot row loaded by its
// two lanes, half each): one 8-byte and four 16-byte shared loads per 16
// products.  Cross terms sum in 32 bits: m <= 64 products of at most
// 4P * P < 2^26 stay below 2^32.
__device__ __forceinline__ void seed_range(const Geometry &g, const EpiConst &ec, const RangeInfo *ri,
                                           const DomainInfo *di, const float4 *dconst, const uint16_t *bblk,
                                           const uint16_t *qblk, int *tbest, int r, int lane, int *bk, uint2 *q2)
{
    const int h = lane >> 4, sl = lane & 15;
    int d;
    if (sl < 9) {
        const int ry = (r / g.nx) * g.n, rx = (r % g.nx) * g.n;
        const int v0 = min(max((ry - g.n / 2) / g.t, 0), g.V - 1);
        const int u0 = min(max((rx - g.n / 2) / g.t, 0), g.U - 1);
        const int v = min(max(v0 + sl / 3 - 1, 0), g.V - 1);
        const int u = min(max(u0 + sl % 3 - 1, 0), g.U - 1);
        d = v * g.U + u;
    } else {
        d = (int)(((long long)r * 2654435761LL + (long long)(sl - 9) * 40503LL) % g.D);
    }
    // every load issued together
    int bv[2];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int i = lane + 32 * j;
        bv[j] = i < g.m ? (int)bblk[(size_t)r * g.m + i] : 0;
    }
    const uint4 *qrow = reinterpret_cast<const uint4 *>(qblk + (size_t)d * g.m);
    const int nv = g.m >> 3;  // 16-byte vectors of a domain row, <= 8
    uint4 qv[4];              // vectors 2 v + h of the slot's row
#pragma unroll
    for (int v = 0; v < 4; ++v) qv[v] = 2 * v + h < nv ? __ldg(qrow + 2 * v + h) : make_uint4(0, 0, 0, 0);
    const RangeInfo rin = ri[r];
    const DomainInfo dd = di[d];
    const float4 c4 = dconst[d];
    const int bp = g.m + 4;  // bk row pitch (ints)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int i = lane + 32 * j;
        if (i < g.m) {
            const int y = i >> g.ln, x = i & (g.n - 1);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                int sy, sx;
                sym_src(k, g.n, y, x, sy, sx);
                bk[k * bp + (sy << g.ln) + sx] = bv[j];
            }
        }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int vv = 2 * v + h;
        if (vv < nv) {
            q2[(2 * vv + 0) * 16 + sl] = make_uint2(qv[v].x, qv[v].y);
            q2[(2 * vv + 1) * 16 + sl] = make_uint2(qv[v].z, qv[v].w);
        }
    }
    __syncwarp();
    const int *bkh = bk + 4 * h * bp;
    uint32_t X[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) X[k] = 0;
    for (int pp = 0; pp < (g.m >> 2); ++pp) {
        const uint2 w = q2[pp * 16 + sl];  // the two halves of a slot read the same words
        const uint32_t qa = w.x & 0xffffu, qb = w.x >> 16, qc = w.y & 0xffffu, qd = w.y >> 16;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int4 b4 = *reinterpret_cast<const int4 *>(bkh + k * bp + 4 * pp);
            X[k] += qa * (uint32_t)b4.x + qb * (uint32_t)b4.y + qc * (uint32_t)b4.z + qd * (uint32_t)b4.w;
        }
    }
    const RangeEpi re = range_epi(rin, ec);
    const long long sqsb = dd.Sq * rin.Sb;
    int best = 0x7fffffff;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const long long num = (long long)g.m * (long long)X[k] - sqsb;  // exact
        const float Xt = __ll2float_rn(num) * ec.invm;
        float rho;
        const float c = epi_code(Xt, c4.x, 0.5f, ec, rho);
        if (fabsf(rho) > re.rho_lim) continue;
        const float ostar = (re.Sb - c * c4.w * ec.inv4ls) * ec.invm;
        if (!(ostar < ec.pmax)) continue;
        best = min(best, f2ord(epi_key(Xt, -0.0f, c, re.zb, c4, ec)));
    }
    best = __reduce_min_sync(0xffffffffu, best);
    if (lane == 0 && best != 0x7fffffff) atomicMin(tbest + r, best);
}

// Compaction (blocks 0 and 1: ranges, domains) and, when seed != 0, the
// seeds (T/32 ranges per block after them) in one launch: both need only the
// statistics, so the seeds run beside the two compaction blocks.
template <int T>
__device__ __forceinline__ void compact_seed_block(const Geometry &g, const EpiConst &ec, int seed,
                                                   const RangeInfo *ri, const DomainInfo *di, const float4 *dconst,
                                                   const uint16_t *bblk, const uint16_t *qblk, const int *rkeep,
                                                   const int *dkeep, int *act, int *dact, int *counts, int *tbest,
                                                   int bx)
{
    extern __shared__ __align__(16) int seed_sm[];
    if (bx < 2) {
        compact_block<T>(g.R, rkeep, act, counts + 0, g.D, dkeep, dact, counts + 2, bx == 1);
        return;
    }
    if (!seed) return;
    // block b takes ranges b, b + nb, b + 2 nb, ...: the screened ranges
    // (which cluster in the image) spread evenly over the blocks
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *bk = seed_sm + warp * seed_warp_ints(g.m);
    if (T == 512) {  // m <= 64: a warp per screened range among the block's 16
        // block b takes ranges b, b + nb, ..., b + 15 nb; its warps take the
        // screened ones in order (every warp reads the 16 keep flags)
        const int nb = (g.R + 15) / 16, b = bx - 2;
        if (b >= nb) return;
        const int rl = lane < 16 ? lane * nb + b : g.R;
        unsigned kept = __ballot_sync(0xffffffffu, rl < g.R && rkeep[rl] != 0);
        if (warp >= __popc(kept)) return;  // warp-uniform
        for (int t = 0; t < warp; ++t) kept &= kept - 1;
        const int r = (__ffs(kept) - 1) * nb + b;
        seed_range(g, ec, ri, di, dconst, bblk, qblk, tbest, r, lane, bk,
                   reinterpret_cast<uint2 *>(bk + 8 * (g.m + 4)));
    } else {
        const int nb = (g.R + T / 32 - 1) / (T / 32);
        if (bx - 2 >= nb) return;
        const int r = warp * nb + (bx - 2);
        if (r >= g.R) return;
        seed_warp<kMaxM / 32>(g, ec, ri, di, dconst, bblk, qblk, rkeep, tbest, r, lane, bk,
                              reinterpret_cast<uint32_t *>(bk + 8 * g.m));
    }
}

template <int T>
__global__ void __launch_bounds__(T, T == 512 ? 2 : 1) k_compact_seed(Geometry g, EpiConst ec, int seed, const RangeInfo *ri,
                                                    const DomainInfo *di, const float4 *dconst,
                                                    const uint16_t *bblk, const uint16_t *qblk, const int *rkeep,
                                                    const int *dkeep, int *act, int *dact, int *counts, int *tbest)
{
    grid_dep_sync();
    compact_seed_block<T>(g, ec, seed, ri, di, dconst, bblk, qblk, rkeep, dkeep, act, dact, counts, tbest,
                          blockIdx.x);
}

template <int T>
__global__ void __launch_bounds__(T, T == 512 ? 2 : 1) k_compact_seed_batch(const SliceCtx *__restrict__ ctx)
{
    grid_dep_sync();
    const SliceCtx &c = ctx[blockIdx.y];
    const EncBufs &b = c.b;
    const CompactBufs &cb = b.cb;
    compact_seed_block<T>(c.g, c.ec, 1, b.ri, b.di, b.dconst, b.bblk, b.qblk, cb.rkeep, cb.dkeep, cb.act, cb.dact,
                          cb.counts, b.tbest, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Compaction, operand rows and seeds in one launch (ranges of at most 8 x 8).
// The statistics kernel left per block a keep mask and its count (block i of
// the ranges covers items i * per .. i * per + per - 1, then the domains'
// blocks).  Every block of this launch prefix-sums those counts itself, so
// the j-th kept range (domain) is found from the sums by a binary search and
// a bit count in its block's mask, and no launch is spent on the compaction:
// the order is the original one, as a stable compaction gives.
constexpr int kRsWarps = 16;             // warps per block (two blocks per SM)
constexpr int kRsMaxStatBlocks = 8192;   // statistics blocks a block can scan

// Shared ints of a block: the seed areas, the prefix sums, scan scratch, the
// items of the block's row units (rounds: an upper bound of the units per
// block and warp, from the largest possible number of kept items) and the
// list of its screened ranges to seed (seeds: the ranges a block owns).
__host__ __device__ constexpr int rows_seed_ints(int m, int nsb, int rounds, int seeds)
{
    return kRsWarps * seed_warp_ints(m) + nsb + 1 + 2 * kRsWarps + 2 + kRsWarps * rounds + seeds;
}

// Position of the t-th (from 0) set bit of x (t < popc(x)).
__device__ __forceinline__ int nth_set_bit(uint32_t x, int t)
{
    int pos = 0;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
        const uint32_t lo = x & ((1u << sh) - 1u);
        const int c = __popc(lo);
        if (t >= c) {
            t -= c;
            x >>= sh;
            pos += sh;
        } else {
            x = lo;
        }
    }
    return pos;
}

// Item of rank j among the kept items of statistics blocks [lo, hi): E holds
// the exclusive prefix sums of the blocks' counts (E[k] <= E[lo] + j <
// E[hi]); per items a block.
__device__ __forceinline__ int kept_item(const int *E, int lo, int hi, int j, const uint4 *bmask, int per)
{
    const int T = E[lo] + j;
    int a = lo, b = hi - 1;  // last k in [lo, hi) with E[k] <= T
    while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (E[mid] <= T) a = mid;
        else b = mid - 1;
    }
    int t = T - E[a];
    const uint4 mk = bmask[a];
    const uint32_t w[4] = {mk.x, mk.y, mk.z, mk.w};
    int base = (a - lo) * per;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int c = __popc(w[k]);
        if (t < c) return base + nth_set_bit(w[k], t);
        t -= c;
        base += 32;
    }
    return -1;  // unreachable when the counts and masks agree
}

template <int LN, bool SPLIT>
__global__ void __launch_bounds__(32 * kRsWarps, 2)
    k_rows_seed(Geometry g, EpiConst ec, int seed, const RangeInfo *ri, const uint16_t *bblk, const DomainInfo *di,
                const uint16_t *qblk, const float4 *dconst, const int *rkeep, const uint4 *bmask,
                const int *bcount, int *tbest, int *act, int *dact, int *counts, float *rs32, __half *ra16,
                float *cb32, __half *cb16, float4 *dconst_c, int *dmap)
{
    extern __shared__ __align__(16) int rs_sm[];
    constexpr int m = 1 << (2 * LN);
    constexpr int per = stats_items(m);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rbs = stats_range_blocks(g), nsb = stats_blocks(g);
    int *wsm = rs_sm + warp * seed_warp_ints(m);  // the warp's seed area, then its row staging
    int *E = rs_sm + kRsWarps * seed_warp_ints(m);
    int *wsum = E + nsb + 1;
    int *first = wsum + 2 * kRsWarps;
    grid_dep_sync();
    // exclusive prefix sums of the statistics blocks' keep counts (each
    // thread a contiguous run of blocks)
    const int run = (nsb + 32 * kRsWarps - 1) / (32 * kRsWarps);
    const int k0 = min(nsb, (int)threadIdx.x * run), k1 = min(nsb, k0 + run);
    int sum = 0;
    for (int k = k0; k < k1; ++k) sum += bcount[k];
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    if (threadIdx.x < 2) first[threadIdx.x] = 0x7fffffff;
    __syncthreads();
    if (warp == 0) {
        const int v = lane < kRsWarps ? wsum[lane] : 0;
        int xs = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, xs, o);
            if (lane >= o) xs += y;
        }
        if (lane < kRsWarps) wsum[kRsWarps + lane] = xs - v;  // exclusive warp offsets
    }
    __syncthreads();
    int acc = wsum[kRsWarps + warp] + x - sum;
    for (int k = k0; k < k1; ++k) {
        E[k] = acc;
        acc += bcount[k];
    }
    if (k1 == nsb && k0 < k1) E[nsb] = acc;
    if (nsb == 0 && threadIdx.x == 0) E[0] = 0;
    __syncthreads();
    const int nr = E[rbs], nd = E[nsb] - E[rbs];
    // the block owns row units u = b kRsWarps + i + k W (i < kRsWarps, warp i
    // takes them); their items (range or domain ids) are found once here, a
    // thread per unit, rather than by each warp per unit
    const int W = gridDim.x * kRsWarps;
    const int T = nr + nd;
    int *items = first + 2;
    int *slist = items + kRsWarps * ((g.R + g.D + W - 1) / W);  // screened ranges to seed
    __shared__ int nseed_s;
    if (seed && warp == 0) {
        // the block's ranges b, b + G, b + 2 G, ...: the screened ones, in order
        int cnt = 0;
        for (int r0 = blockIdx.x; r0 < g.R; r0 += 32 * gridDim.x) {
            const int r = r0 + lane * gridDim.x;
            const bool k = r < g.R && rkeep[r] != 0;
            const unsigned bal = __ballot_sync(0xffffffffu, k);
            if (k) slist[cnt + __popc(bal & ((1u << lane) - 1u))] = r;
            cnt += __popc(bal);
        }
        if (lane == 0) nseed_s = cnt;
    }
    {
        const int u0 = blockIdx.x * kRsWarps;
        const int K = T > u0 ? (T - u0 + W - 1) / W : 0;
        for (int q = threadIdx.x; q < K * kRsWarps; q += blockDim.x) {
            const int u = u0 + (q % kRsWarps) + (q / kRsWarps) * W;
            int it = -1;
            if (u < nr)
                it = kept_item(E, 0, rbs, u, bmask, per);
            else if (u < T)
                it = kept_item(E, rbs, nsb, u - nr, bmask, per);
            items[q] = it;
        }
    }
    __syncthreads();
    if (blockIdx.x == 0) {
        // the first range (domain) that is not kept, as the compaction
        // reports it: blocks whose count is below their valid items
        for (int k = threadIdx.x; k < nsb; k += blockDim.x) {
            const bool dom = k >= rbs;
            const int lo_item = (dom ? k - rbs : k) * per;
            const int valid = min(per, (dom ? g.D : g.R) - lo_item);
            if (bcount[k] < valid) {
                const uint4 mk = bmask[k];
                const uint32_t w[4] = {mk.x, mk.y, mk.z, mk.w};
                int f = -1;
                for (int q = 0; q < 4 && f < 0; ++q) {
                    const int nv = min(32, valid - 32 * q);
                    if (nv <= 0) break;
                    const uint32_t vm = nv >= 32 ? 0xffffffffu : ((1u << nv) - 1u);
                    const uint32_t z = ~w[q] & vm;
                    if (z) f = 32 * q + __ffs(z) - 1;
                }
                if (f >= 0) atomicMin(first + (dom ? 1 : 0), lo_item + f);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            counts[0] = nr;
            counts[1] = first[0] == 0x7fffffff ? -1 : first[0];
            counts[2] = nd;
            counts[3] = first[1] == 0x7fffffff ? -1 : first[1];
        }
    }
    // seeds: the block's screened ranges (listed above), warp w takes
    // entries w, w + kRsWarps, ...
    if (seed) {
        const int ns = nseed_s;
        for (int e = warp; e < ns; e += kRsWarps) {
            __syncwarp();  // the warp's previous seed area is read
            seed_range(g, ec, ri, di, dconst, bblk, qblk, tbest, slist[e], lane, wsm,
                       reinterpret_cast<uint2 *>(wsm + 8 * (m + 4)));
        }
        __syncwarp();  // the seed area becomes the row staging
    }
    // operand rows: warp units over the grid, the kept ranges' rows first
    const RowLane rl = row_lane<LN>(lane);
    uint16_t *st = reinterpret_cast<uint16_t *>(wsm);
    for (int k = 0;; ++k) {
        const int u = blockIdx.x * kRsWarps + warp + k * W;
        if (u >= T) break;
        const int it = items[k * kRsWarps + warp];
        if (it < 0) continue;  // unreachable: counts and masks come from one statistics launch
        if (u < nr) {
            const int r = it;
            if (lane == 0) act[u] = r;
            range_row<LN, SPLIT>(ri, bblk, u, r, lane, rs32, ra16);
        } else {
            const int j = u - nr;
            const int d = it;
            if (lane == 0) dact[j] = d;
            __syncwarp();  // the staging of the warp's previous domain is read
            domain_rows_warp<LN, SPLIT>(di, qblk, dconst, j, d, lane, rl, st, cb32, cb16, dconst_c, dmap);
        }
    }
}

// The fused kernels of a geometry (ranges of at most 8 x 8).
template <typename Launch>
static cudaError_t with_rows_seed_kernel(const Geometry &g, Launch &&launch)
{
    const bool sp = g.split_hilo != 0;
    switch (g.ln) {
    case 2: return sp ? launch(k_rows_seed<2, true>) : launch(k_rows_seed<2, false>);
    case 3: return sp ? launch(k_rows_seed<3, true>) : launch(k_rows_seed<3, false>);
    default: return cudaErrorInvalidValue;
    }
}

// Launch shape of the compaction + seed launch: T/32 seeded ranges per block.
template <typename Launch>
static cudaError_t with_seed_shape(int m, Launch &&launch)
{
    if (seed_warps(m) == 16) {
        cudaError_t e = cudaFuncSetAttribute(k_compact_seed<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)seed_smem(m));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_compact_seed_batch<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)seed_smem(m));
        return e != cudaSuccess ? e : launch(k_compact_seed<512>, k_compact_seed_batch<512>, 512);
    }
    cudaError_t e = cudaFuncSetAttribute(k_compact_seed<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)seed_smem(m));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_compact_seed_batch<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)seed_smem(m));
    return e != cudaSuccess ? e : launch(k_compact_seed<256>, k_compact_seed_batch<256>, 256);
}

// SMs of the current device (queried once).
static int prep_sms()
{
    static int n = 0;
    if (n <= 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) ==
                                                     cudaSuccess && v > 0)
            n = v;
        else
            return 1;
    }
    return n;
}

cudaError_t launch_prep(const Geometry &g, const void *img, const EpiConst &ec, int dense, int tc_mode,
                        const int *active,
                        RangeInfo *ri, DomainInfo *di, float4 *dconst, uint16_t *bblk, uint16_t *qblk, float *rs32,
                        float *cb32, __half *ra16, __half *cb16, int *tbest, const CompactBufs &cb, int *zero4,
                        int seed, cudaStream_t st)
{
    const int rb = (g.R + 7) / 8, db = (g.D + 7) / 8;
    const int nsb = stats_blocks(g);
    // ranges of at most 8 x 8 (the seed's shared memory per warp is small
    // there) and statistics blocks whose counts fit a block's shared memory:
    // compaction, operand rows and seeds in one launch after the statistics
    const bool fused = g.m <= 64 && nsb <= kRsMaxStatBlocks && cb.bmask;
    cudaError_t e = with_stats_kernel(g, [&](auto one, auto) {
        return launch_dep(one, dim3(nsb), dim3(256), 0, st, g, ec, img, dense, tc_mode, active, ri, bblk, tbest, di,
                          dconst, qblk, cb.rkeep, cb.dkeep, zero4, fused ? cb.bmask : nullptr,
                          fused ? cb.bcount : nullptr);
    });
    if (e != cudaSuccess) return e;
    if (fused) {
        // one wave: the resident blocks (two per SM)
        const int blocks = 2 * prep_sms();
        const int W = blocks * kRsWarps;
        const int rounds = (g.R + g.D + W - 1) / W;  // row units a warp takes, at most
        const int seeds = (g.R + blocks - 1) / blocks;  // ranges a block owns
        const size_t smem = sizeof(int) * (size_t)rows_seed_ints(g.m, nsb, rounds, seeds);
        return with_rows_seed_kernel(g, [&](auto kern) {
            cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e2 != cudaSuccess) return e2;
            return launch_dep(kern, dim3(blocks), dim3(32 * kRsWarps), smem, st, g, ec, seed, (const RangeInfo *)ri,
                              (const uint16_t *)bblk, (const DomainInfo *)di, (const uint16_t *)qblk,
                              (const float4 *)dconst, (const int *)cb.rkeep, (const uint4 *)cb.bmask,
                              (const int *)cb.bcount, tbest, cb.act, cb.dact, cb.counts, rs32, ra16, cb32, cb16,
                              cb.dconst_c, cb.dmap);
        });
    }
    const int sw = seed_warps(g.m);
    e = with_seed_shape(g.m, [&](auto one, auto, int threads) {
        const int per = sw;  // ranges per seed block
        return launch_dep(one, dim3(2 + (seed ? (g.R + per - 1) / per : 0)), dim3(threads), seed ? seed_smem(g.m) : 0,
                          st, g, ec, seed, (const RangeInfo *)ri, (const DomainInfo *)di, (const float4 *)dconst,
                          (const uint16_t *)bblk, (const uint16_t *)qblk, (const int *)cb.rkeep,
                          (const int *)cb.dkeep, cb.act, cb.dact, cb.counts, tbest);
    });
    if (e != cudaSuccess) return e;
    const int blocks = std::max(1, std::min(rb + db, rows_blocks_per_sm(g.ln) * prep_sms()));
    return with_rows_kernel(g, [&](auto one, auto) {
        return launch_dep(one, dim3(blocks), dim3(256), 0, st, (const RangeInfo *)ri, (const uint16_t *)bblk,
                          (const DomainInfo *)di, (const uint16_t *)qblk, (const float4 *)dconst, (const int *)cb.act,
                          (const int *)cb.dact, (const int *)cb.counts, rs32, ra16, cb32, cb16, cb.dconst_c, cb.dmap);
    });
}

// Batched prep stages of n slices (ctx: device array; blocks / ranges: the
// largest slice's, so a group of equal slices wastes no blocks).
int stats_grid(const Geometry &g) { return stats_blocks(g); }

cudaError_t launch_stats_batch(const Geometry &g, const SliceCtx *ctx, int n, int blocks, int dense, int tc_mode,
                               cudaStream_t st)
{
    return with_stats_kernel(
        g, [&](auto, auto many) { return launch_dep(many, dim3(blocks, n), dim3(256), 0, st, ctx, dense, tc_mode); });
}

// ranges, m: the largest of the slices' ranges and their common block size
cudaError_t launch_compact_seed_batch(const SliceCtx *ctx, int n, int ranges, int m, cudaStream_t st)
{
    const int sw = seed_warps(m);
    return with_seed_shape(m, [&](auto, auto many, int threads) {
        const int per = sw;  // ranges per seed block
        return launch_dep(many, dim3(2 + (ranges + per - 1) / per, n), dim3(threads), seed_smem(m), st, ctx);
    });
}

// g: the geometry of the group's slices (range size and bit depth are
// common to all slices of a batch)
cudaError_t launch_rows_batch(const Geometry &g, const SliceCtx *ctx, int n, int blocks, cudaStream_t st)
{
    const int x = std::max(1, std::min(blocks, rows_blocks_per_sm(g.ln) * prep_sms() / std::max(1, n)));
    return with_rows_kernel(g, [&](auto, auto many) { return launch_dep(many, dim3(x, n), dim3(256), 0, st, ctx); });
}



}  // namespace fic
