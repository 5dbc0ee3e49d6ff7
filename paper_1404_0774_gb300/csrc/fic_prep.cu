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

// One thread per range: statistics, centre, operand rows.
__global__ void k_range_prep(Geometry g, EpiConst ec, const void *img, RangeInfo *ri, uint16_t *bblk,
                             float *rs32, __half *ra16, int *tbest)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= g.R) return;
    const int ry = (r / g.nx) * g.n, rx = (r % g.nx) * g.n;
    long long Sb = 0, Sbb = 0;
    int bmin = 1 << 30, bmax = -1;
    for (int i = 0; i < g.m; ++i) {
        const int y = i / g.n, x = i % g.n;
        const int b = load_px(img, g.B, (size_t)(ry + y) * g.pitch + rx + x);
        Sb += b;
        Sbb += (long long)b * b;
        bmin = min(bmin, b);
        bmax = max(bmax, b);
        bblk[(size_t)r * g.m + i] = (uint16_t)b;
    }
    // centre: nearest integer to the mean, kept within 2048 of every pixel so
    // that b - c_r is an exact FP16 integer
    long long cr = (2 * Sb + g.m) / (2 * (long long)g.m);
    cr = max((long long)(bmax - 2048), min((long long)(bmin + 2048), cr));
    const int c_r = (int)cr;
    const int e_r = (int)(Sb - (long long)g.m * c_r);
    double bp2 = 0.0;
    for (int i = 0; i < g.m; ++i) {
        const int y = i / g.n, x = i % g.n;
        const int bc = load_px(img, g.B, (size_t)(ry + y) * g.pitch + rx + x) - c_r;
        bp2 += (double)bc * bc;
        if (rs32) rs32[(size_t)r * g.m + i] = (float)bc;
        if (ra16) {
            ra16[(size_t)r * g.KP + i] = __int2half_rn(bc);
            if (g.split_hilo) ra16[(size_t)r * g.KP + g.m + i] = __int2half_rn(bc);
        }
    }
    if (ra16) {
        const int base = g.split_hilo ? 2 * g.m : g.m;
        const int e_hi = (e_r >= 0) ? (e_r >> 10) : -((-e_r + 1023) >> 10);
        const int e_lo = e_r - 1024 * e_hi;
        for (int j = base; j < g.KP; ++j) ra16[(size_t)r * g.KP + j] = __float2half_rn(0.0f);
        ra16[(size_t)r * g.KP + base] = __int2half_rn(e_hi);
        ra16[(size_t)r * g.KP + base + 1] = __int2half_rn(e_lo);
    }
    RangeInfo info;
    info.Sb = Sb;
    info.Sbb = Sbb;
    info.c_r = c_r;
    info.e_r = e_r;
    info.sbbc = (float)((double)((long long)g.m * Sbb - Sb * Sb) / g.m);
    const double z = 4.0 * g.Ls * (double)Sb;
    info.zb = (float)(g.mod_g ? fmod(z, g.G) : z);
    info.bp2 = (float)bp2;
    // FP32 error of Ls*s: ~1e-6 when the cross term is exact, plus the
    // accumulation error of high-variance pairs (grows with sum (b-c_r)^2)
    const double eta = 1e-5 + 12.0 * g.Ls * 64.0 * bp2 * 3.552713678800501e-15;  // 2^-48
    info.rho_lim = (float)(0.5 - fmin(eta, 0.25));
    // Screening allowance.  A candidate within reach of the winner has
    // |c| * sqrt(sum (q-q_mean)^2) <= 4*Ls*(sqrt(Sbb_c) + sqrt(R)), R <= Eb; its
    // centred products (hi/lo split included) then sum to at most S.  Below
    // 2^23 every FP32 partial sum of integers is exact and the cross term
    // carries no error; otherwise allow 2^-15 relative.
    const double sbbc = fmax((double)info.sbbc, 0.0);
    const double Eb = 4.0 * (sbbc + ec.delta_o);
    const double sb = sqrt(bp2);
    const double S = (4.0 * g.Ls * (sqrt(sbbc) + sqrt(Eb)) + sqrt((double)g.m)) * sb +
                     (g.split_hilo ? 128.0 * sqrt((double)g.m) * sb : 0.0);
    const bool exact = S < 8388608.0;
    const double gam = 3.0517578125e-05;  // 2^-15
    info.beta_q = exact ? 0.0f : (float)(4.0 * g.Ls * gam * sb);
    info.beta_a = (float)(3.814697265625e-06 * 2.0 * g.Ls * (sbbc + ec.delta_o) + 1e-3 +
                          (exact ? 0.0 : gam * g.Ls * 128.0 * sqrt((double)g.m) * sb));
    info.shadow = bmin == bmax ? 1 : 0;
    info.pad = 0;
    tbest[r] = 0x7f800000;  // +inf in the ordered-integer encoding of floats
    ri[r] = info;
}

// One block of m threads per domain.
__global__ void k_domain_prep(Geometry g, const void *img, DomainInfo *di, float4 *dconst,
                              uint16_t *qblk, float *cb32, __half *cb16)
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
        float4 c4;
        c4.x = den > 0 ? (float)(2.0 * m / (double)den) : 0.0f;
        c4.y = (float)(g.mod_g ? fmod((double)Sq, g.G) : (double)Sq);
        c4.z = (float)((double)den / (8.0 * m * g.Ls));
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
    if (!live) return;
    // candidate rows 8d+k: output pixel (y,x) of S_k(tau(d)) reads q at sym_src
    for (int k = 0; k < 8; ++k) {
        int sy, sx;
        sym_src(k, n, y, x, sy, sx);
        const int qc = q_s[sy * n + sx] - c_d;
        const size_t row = (size_t)d * 8 + k;
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
            if (i < g.KP - (g.split_hilo ? 2 * m : m)) {
                const int base = g.split_hilo ? 2 * m : m;
                float v = 0.0f;
                if (i == 0) v = -1024.0f * (float)fd_s / (float)m;
                if (i == 1) v = -(float)fd_s / (float)m;
                rowp[base + i] = __float2half_rn(v);
            }
        }
    }
}

cudaError_t launch_prep(const Geometry &g, const void *img, const EpiConst &ec, RangeInfo *ri, DomainInfo *di,
                        float4 *dconst, uint16_t *bblk, uint16_t *qblk, float *rs32, float *cb32,
                        __half *ra16, __half *cb16, int *tbest, cudaStream_t st)
{
    k_range_prep<<<(g.R + 127) / 128, 128, 0, st>>>(g, ec, img, ri, bblk, rs32, ra16, tbest);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_domain_prep<<<g.D, g.m < 32 ? 32 : g.m, 0, st>>>(g, img, di, dconst, qblk, cb32, cb16);
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
    const int r = blockIdx.x;
    const int s = threadIdx.x;  // 256 seed slots
    const RangeInfo rin = ri[r];
    if (rin.shadow) return;
    const int slot_d = s >> 3, k = s & 7;
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
    long long X = 0;
    for (int i = 0; i < g.m; ++i) {
        int sy, sx;
        sym_src(k, g.n, i / g.n, i % g.n, sy, sx);
        X += (long long)qblk[(size_t)d * g.m + sy * g.n + sx] * bblk[(size_t)r * g.m + i];
    }
    const DomainInfo dd = di[d];
    const float Xt = (float)((double)((long long)g.m * X - dd.Sq * rin.Sb) / g.m);
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
