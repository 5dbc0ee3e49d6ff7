// Differentiable refinement: the decoder with real-valued (FP32) contrast s
// and offset o per range, unrolled for T iterations, and its adjoint.
//
// Forward (the decoder of the abstract / Section VI, Jacobi form, no clamp):
//   x_{t+1}[p] = s_r * a_t[p] + o_r   for every pixel p of range r,
//   a_t[p] = (1/4) * (sum of the 2x2 source pixels of x_t that S_k places at p),
// from a flat x_0.  Loss: L = (1/N) sum_p (x_T[p] - I[p])^2.
// Adjoint, in reverse (g_T = dL/dx_T = 2 (x_T - I) / N):
//   dL/ds_r += sum_{p in r} g_{t+1}[p] a_t[p],   dL/do_r += sum_{p in r} g_{t+1}[p],
//   g_t[q] = sum over the output pixels p that read source pixel q of s_r/4 g_{t+1}[p].
// The transpose of the gather is formed as a gather too (no atomics, a fixed
// summation order): source pixel q lies in the domains whose 2n x 2n window
// covers it, and every range using such a domain reads q at exactly one of its
// pixels (S_k is a bijection), found through a domain -> ranges index built
// once per set of maps.  Iterates are checkpointed every second step; the odd
// ones are recomputed from the even ones during the reverse sweep.
#include <algorithm>

#include "fic_internal.cuh"

namespace fic {

namespace {

// S_k inverse: rot90 and rot270 swap, every other symmetry is an involution
__device__ __forceinline__ int sym_inverse(int k) { return k == 1 ? 3 : (k == 3 ? 1 : k); }

__device__ __forceinline__ float load_ref(const void *img, int B, size_t off)
{
    return B <= 8 ? (float)((const uint8_t *)img)[off] : (float)((const uint16_t *)img)[off];
}

}  // namespace

// Per range: offset of its domain's top-left pixel, symmetry; domain use counts.
__global__ void k_ref_ranges(RefineGeo rg, const fic_map *maps, int *roff, int *rsym, int *dcount)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rg.R) return;
    const int d = (int)maps[r].domain_idx, k = maps[r].iso;
    roff[r] = (d / rg.U) * rg.t * rg.w + (d % rg.U) * rg.t;
    rsym[r] = k;
    if (dcount) atomicAdd(dcount + d, 1);
}

// Exclusive scan of the D domain counts (one block), off[D] = total.
__global__ void __launch_bounds__(1024) k_ref_scan(int D, const int *cnt, int *off, int *cursor)
{
    __shared__ int wsum[32];
    __shared__ int base_s;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) base_s = 0;
    __syncthreads();
    for (int i0 = 0; i0 < D; i0 += 1024) {
        const int i = i0 + t;
        const int v = i < D ? cnt[i] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            const int u = wsum[lane];
            int z = u;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, z, o);
                if (lane >= o) z += y;
            }
            wsum[lane] = z - u;
        }
        __syncthreads();
        const int base = base_s;
        if (i < D) {
            off[i] = base + wsum[w] + x - v;
            cursor[i] = 0;
        }
        __syncthreads();
        if (t == 1023) base_s = base + wsum[31] + x;
        __syncthreads();
    }
    if (t == 0) off[D] = base_s;
}

// Ranges of each domain (CSR rows in range order), one block: ranges are taken
// 1024 at a time; a range's slot is its domain's row start, plus the ranges of
// that domain in earlier rounds (cursor), plus those earlier in this round.
__global__ void __launch_bounds__(1024) k_ref_fill(int R, const fic_map *maps, const int *off, int *cursor, int *rng)
{
    __shared__ int d_s[1024];
    const int t = threadIdx.x;
    for (int r0 = 0; r0 < R; r0 += 1024) {
        const int r = r0 + t;
        const int d = r < R ? (int)maps[r].domain_idx : -1;
        d_s[t] = d;
        __syncthreads();
        if (r < R) {
            int rank = 0;
            for (int u = 0; u < t; ++u) rank += d_s[u] == d;
            rng[off[d] + cursor[d] + rank] = r;
        }
        __syncthreads();  // every slot of this round is placed before the cursors move
        if (r < R) atomicAdd(cursor + d, 1);
        __syncthreads();
    }
}

// Work items of the adjoint's per-domain sums: each domain's users split into
// runs of at most kAdjRun (in range order).  nitem[d] = ceil(users / kAdjRun).
constexpr int kAdjRun = 32;
__global__ void k_ref_item_count(int D, const int *off, int *nitem)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d < D) nitem[d] = (off[d + 1] - off[d] + kAdjRun - 1) / kAdjRun;
}

__global__ void k_ref_item_fill(int D, const int *off, const int *ioff, int4 *items)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= D) return;
    const int b = off[d], e = off[d + 1];
    for (int i = 0, u = b; u < e; ++i, u += kAdjRun) items[ioff[d] + i] = make_int4(d, u, min(e, u + kAdjRun), 0);
}

// x1 = W(x0): thread per pixel.
__global__ void k_ref_step(RefineGeo rg, const int *roff, const int *rsym, const float *s, const float *o,
                           const float *x0, float *x1)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= rg.w * rg.h) return;
    const int y = p / rg.w, x = p - (p / rg.w) * rg.w;
    const int r = (y >> rg.ln) * rg.nx + (x >> rg.ln);
    const int li = sym_src_index(sym_flags(rsym[r], rg.n), rg.ln, y & (rg.n - 1), x & (rg.n - 1));
    const int q = roff[r] + 2 * (li >> rg.ln) * rg.w + 2 * (li & (rg.n - 1));
    const float a = 0.25f * (x0[q] + x0[q + 1] + x0[q + rg.w] + x0[q + rg.w + 1]);
    x1[p] = fmaf(s[r], a, o[r]);
}

// g = 2 (x - I) / N and per-block partial sums of (x - I)^2 (FP64, fixed order).
__global__ void __launch_bounds__(256) k_ref_loss(RefineGeo rg, const float *x, const void *img, int B, int pitch,
                                                  float *g, double *partial)
{
    __shared__ double red[8];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int N = rg.w * rg.h;
    double se = 0.0;
    if (p < N) {
        const int y = p / rg.w, xx = p - (p / rg.w) * rg.w;
        const float d = x[p] - load_ref(img, B, (size_t)y * pitch + xx);
        g[p] = 2.0f * d / (float)N;
        se = (double)d * (double)d;
    }
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = se;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += red[i];
        partial[blockIdx.x] = t;
    }
}

// loss[step] = sum of the partials / N (one block, fixed order); step counter += 1.
__global__ void __launch_bounds__(1024) k_ref_loss_final(int nb, int N, const double *partial, float *loss, int *step,
                                                         int advance)
{
    __shared__ double red[32];
    double t = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) t += partial[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tt = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tt += red[w];
        if (loss) loss[*step] = (float)(tt / (double)N);
        if (advance) *step += 1;
    }
}

// dL/ds_r, dL/do_r contributions of one reverse step: warp per range.
__global__ void k_ref_grad_range(RefineGeo rg, const int *roff, const int *rsym, const float *xt, const float *g1,
                                 float *ds, float *dof, int first)
{
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rg.R) return;
    const int ry = (r / rg.nx) * rg.n, rx = (r - (r / rg.nx) * rg.nx) * rg.n;
    const SymFlags sf = sym_flags(rsym[r], rg.n);
    float gs = 0.0f, go = 0.0f;
    for (int i = lane; i < rg.n * rg.n; i += 32) {
        const int y = i >> rg.ln, x = i & (rg.n - 1);
        const int li = sym_src_index(sf, rg.ln, y, x);
        const int q = roff[r] + 2 * (li >> rg.ln) * rg.w + 2 * (li & (rg.n - 1));
        const float a = 0.25f * (xt[q] + xt[q + 1] + xt[q + rg.w] + xt[q + rg.w + 1]);
        const float gp = g1[(ry + y) * rg.w + rx + x];
        gs = fmaf(gp, a, gs);
        go += gp;
    }
    for (int o = 16; o > 0; o >>= 1) {
        gs += __shfl_xor_sync(0xffffffffu, gs, o);
        go += __shfl_xor_sync(0xffffffffu, go, o);
    }
    if (lane == 0) {  // the first reverse step starts the sums
        ds[r] = first ? gs : ds[r] + gs;
        dof[r] = first ? go : dof[r] + go;
    }
}

// g0 = W'^T g1 in three gathers (no atomics, fixed summation order).
// 1. Per work item (a run of <= 32 users of one domain): partial[i][j] = sum
//    over its ranges r (in order) of s_r * g1[the pixel of r that reads
//    contracted pixel j] (S_k is a bijection, so that pixel is unique).
__global__ void __launch_bounds__(256) k_ref_adj_items(RefineGeo rg, const int4 *items, const int *n_items,
                                                       const int *rng, const int *rsym, const float *s,
                                                       const float *g1, float *partial)
{
    const int m = rg.n * rg.n, lm = 2 * rg.ln;
    const int per = 256 >> lm > 0 ? 256 >> lm : 1;  // items per block
    const int it = blockIdx.x * per + (threadIdx.x >> lm);
    const int j = threadIdx.x & (m - 1);
    if ((threadIdx.x >> lm) >= per || it >= *n_items) return;
    for (int jj = j; jj < m; jj += 256) {  // m = 256: one item per block, each thread one pixel
        const int4 w = items[it];
        float acc = 0.0f;
        for (int u = w.y; u < w.z; ++u) {
            const int r = rng[u];
            const int li = sym_src_index(sym_flags(sym_inverse(rsym[r]), rg.n), rg.ln, jj >> rg.ln, jj & (rg.n - 1));
            const int ry = (r / rg.nx) * rg.n, rx = (r - (r / rg.nx) * rg.nx) * rg.n;
            acc = fmaf(s[r], g1[(ry + (li >> rg.ln)) * rg.w + rx + (li & (rg.n - 1))], acc);
        }
        partial[(size_t)it * m + jj] = acc;
    }
}

// 2. Per domain: C_d[j] = sum of its items' partials in item order (0 when unused).
__global__ void k_ref_adj_domain(RefineGeo rg, const int *ioff, const float *partial, float *C)
{
    const int m = rg.n * rg.n;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rg.D * m) return;
    const int d = idx / m, j = idx - (idx / m) * m;
    float t = 0.0f;
    for (int i = ioff[d]; i < ioff[d + 1]; ++i) t += partial[(size_t)i * m + j];
    C[idx] = t;
}

// 3. Per source pixel q: g0[q] = 1/4 * sum over the domains whose 2n x 2n
//    window covers q (in domain order) of C_d at q's contracted pixel.
__global__ void k_ref_adj_pixel(RefineGeo rg, const float *C, float *g0)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= rg.w * rg.h) return;
    const int qy = q / rg.w, qx = q - (q / rg.w) * rg.w;
    const int n2 = 2 * rg.n, m = rg.n * rg.n;
    // domains u with u*t <= qx < u*t + 2n
    const int u0 = max(0, (qx - n2 + rg.t) / rg.t), u1 = min(rg.U - 1, qx / rg.t);
    const int v0 = max(0, (qy - n2 + rg.t) / rg.t), v1 = min(rg.V - 1, qy / rg.t);
    float acc = 0.0f;
    for (int v = v0; v <= v1; ++v)
        for (int u = u0; u <= u1; ++u) {
            const int a = (qy - v * rg.t) >> 1, b = (qx - u * rg.t) >> 1;  // contracted pixel of the domain
            acc += C[(size_t)(v * rg.U + u) * m + (a << rg.ln) + b];
        }
    g0[q] = 0.25f * acc;
}

// Adam on theta = (s, o / P) with gradients (dL/ds, P dL/do); step counter
// already advanced (bias corrections use it).
__global__ void k_ref_adam(int R, float *s, float *o, const float *ds, const float *dof, float *m, float *v,
                           const int *step, float lr, float P)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * R) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const int t = *step;
    const bool is_s = i < R;
    const int r = is_s ? i : i - R;
    const float g = is_s ? ds[r] : P * dof[r];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.0f - powf(b1, (float)t));
    const float vh = vi / (1.0f - powf(b2, (float)t));
    const float upd = lr * mh / (sqrtf(vh) + eps);
    if (is_s) s[r] -= upd;
    else o[r] -= upd * P;
}

__global__ void k_ref_fill_f(int n, float v, float *a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// ---------------------------------------------------------------- launches

namespace {
inline int blocks(long long n, int t) { return (int)((n + t - 1) / t); }
}  // namespace

cudaError_t refine_ranges(const RefineGeo &rg, const fic_map *maps, const RefineBufs &b, bool with_index,
                          cudaStream_t st)
{
    cudaError_t e;
    if (with_index && (e = cudaMemsetAsync(b.dcount, 0, sizeof(int) * rg.D, st)) != cudaSuccess) return e;
    k_ref_ranges<<<blocks(rg.R, 256), 256, 0, st>>>(rg, maps, b.roff, b.rsym, with_index ? b.dcount : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess || !with_index) return e;
    k_ref_scan<<<1, 1024, 0, st>>>(rg.D, b.dcount, b.doff, b.cursor);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_ref_fill<<<1, 1024, 0, st>>>(rg.R, maps, b.doff, b.cursor, b.drng);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_ref_item_count<<<blocks(rg.D, 256), 256, 0, st>>>(rg.D, b.doff, b.nitem);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_ref_scan<<<1, 1024, 0, st>>>(rg.D, b.nitem, b.ioff, b.cursor);  // ioff[D] = number of items
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_ref_item_fill<<<blocks(rg.D, 256), 256, 0, st>>>(rg.D, b.doff, b.ioff, b.items);
    return cudaGetLastError();
}

cudaError_t refine_forward(const RefineGeo &rg, const RefineBufs &b, const float *s, const float *o, float init,
                           int iters, float *ckpt, float *x_out, cudaStream_t st)
{
    const int N = rg.w * rg.h;
    // x_0 in checkpoint 0; x_{t+1} computed from x_t; even t kept in ckpt[t/2]
    k_ref_fill_f<<<blocks(N, 256), 256, 0, st>>>(N, init, ckpt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float *cur = ckpt;
    for (int t = 0; t < iters; ++t) {
        float *nxt = (t + 1 == iters) ? x_out : ((t + 1) % 2 == 0 ? ckpt + (size_t)((t + 1) / 2) * N : b.tmp);
        k_ref_step<<<blocks(N, 256), 256, 0, st>>>(rg, b.roff, b.rsym, s, o, cur, nxt);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cur = nxt;
    }
    return cudaSuccess;
}

cudaError_t refine_backward(const RefineGeo &rg, const RefineBufs &b, const float *s, const float *o, int iters,
                            const float *ckpt, const float *grad_x, float *ds, float *dof, cudaStream_t st)
{
    const int N = rg.w * rg.h;
    cudaError_t e;
    const float *g1 = grad_x;
    for (int t = iters - 1; t >= 0; --t) {
        const float *xt;
        if (t % 2 == 0) {
            xt = ckpt + (size_t)(t / 2) * N;
        } else {  // recompute the odd iterate from the even checkpoint before it
            k_ref_step<<<blocks(N, 256), 256, 0, st>>>(rg, b.roff, b.rsym, s, o, ckpt + (size_t)(t / 2) * N, b.tmp);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            xt = b.tmp;
        }
        k_ref_grad_range<<<blocks(rg.R, 8), 256, 0, st>>>(rg, b.roff, b.rsym, xt, g1, ds, dof, t == iters - 1 ? 1 : 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (t > 0) {
            float *g0 = (g1 == b.g[0]) ? b.g[1] : b.g[0];
            const int m = rg.n * rg.n;
            const int per = std::max(1, 256 / m);
            k_ref_adj_items<<<blocks(rg.R, per), 256, 0, st>>>(rg, b.items, b.ioff + rg.D, b.drng, b.rsym, s, g1,
                                                               b.ipart);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            k_ref_adj_domain<<<blocks((long long)rg.D * m, 256), 256, 0, st>>>(rg, b.ioff, b.ipart, b.C);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            k_ref_adj_pixel<<<blocks(N, 256), 256, 0, st>>>(rg, b.C, g0);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            g1 = g0;
        }
    }
    return cudaSuccess;
}

cudaError_t refine_loss(const RefineGeo &rg, const RefineBufs &b, const float *x, const void *img, int B, int pitch,
                        float *g, float *loss, int advance, cudaStream_t st)
{
    const int N = rg.w * rg.h;
    const int nb = blocks(N, 256);
    k_ref_loss<<<nb, 256, 0, st>>>(rg, x, img, B, pitch, g, b.partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ref_loss_final<<<1, 1024, 0, st>>>(nb, N, b.partial, loss, b.step, advance);
    return cudaGetLastError();
}

cudaError_t refine_adam(const RefineGeo &rg, const RefineBufs &b, float *s, float *o, float lr, float P,
                        cudaStream_t st)
{
    k_ref_adam<<<blocks(2 * rg.R, 256), 256, 0, st>>>(rg.R, s, o, b.ds, b.dof, b.m, b.v, b.step, lr, P);
    return cudaGetLastError();
}

size_t refine_partials(const RefineGeo &rg) { return (size_t)blocks((long long)rg.w * rg.h, 256); }

}  // namespace fic
