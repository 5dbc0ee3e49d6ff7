/*
 * FP64 CPU oracle for PIFS fractal encoding and decoding.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product library
 * never links, includes or calls it, and it shares no code with the CUDA path.
 *
 * What it computes (Haque et al., "GPU Accelerated Fractal Image Compression
 * for Medical Imaging", arXiv 1404.0774):
 *
 *  - Ranges: the image is cut into non-overlapping n x n blocks (Section V,
 *    Section VI).  Range r = j*(W/n) + i has its top-left pixel at (n*j, n*i).
 *  - Domains: overlapping 2n x 2n blocks on a grid of spacing STEP = t
 *    (Section V, Algorithm 1).  Domain d = v*U + u, U = (W-2n)/t + 1, has its
 *    top-left pixel at (t*v, t*u).
 *  - Contraction tau: the fixed domain->range contraction (Section V); read as
 *    the 2x2 mean, a[y][x] = (sum of the 2x2 pixels at (2y, 2x)) / 4.
 *  - Eight symmetries S_k (Section V: rotations by 90/180/270 degrees and
 *    mirroring), numbered k = 0..7 as identity, rot90 cw, rot180, rot270 cw,
 *    mirror left-right, mirror top-bottom, transpose, anti-transpose.
 *  - Least squares (eq 9, eq 10) with the denominator written as the domain
 *    variance n*sum(a^2) - (sum a)^2 that the text after eq 10 states; when it
 *    is zero, s = 0 and o = mean(b) (eq 11, eq 12).
 *  - Quantisation (not in the paper; the workload fixes it): s clamped to
 *    [-1, 1] and rounded half away from zero to c/Ls, Ls = 2^(s_bits-1) - 1;
 *    o is then recomputed from the quantised s as in eq 10, clamped to
 *    [-P, P] (P = 2^B - 1), and rounded to e*P/Lo, Lo = 2^(o_bits-1) - 1.
 *    s_bits = 0 (o_bits = 0) turns quantisation of s (of o) off.
 *  - Residual R = sum_i (s*a_i + o - b_i)^2 (eq 8), summed over the pixels.
 *  - Search (Algorithm 2, per range as in Algorithm 3): domains outer,
 *    symmetries inner, and a candidate replaces the best only if its residual
 *    is strictly smaller, so the first of equal minima (lowest d, then k) wins.
 *  - Decoding: the maps are iterated from a flat start image; every range is
 *    replaced by s * S_k(tau(domain)) + o computed from the previous iterate,
 *    with no clamping inside the iteration; the result is clamped to [0, P].
 *
 * All arithmetic is IEEE double with no contraction (build with
 * -ffp-contract=off), in the order written here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n;         /* range size                       */
    int32_t t;         /* domain grid spacing (STEP)       */
    int32_t bit_depth; /* B, P = 2^B - 1                   */
    int32_t s_bits;    /* 0 = s unquantised                */
    int32_t o_bits;    /* 0 = o unquantised                */
} orc_params;

typedef struct {
    int32_t d, k, c, e; /* domain, symmetry, s code, o code */
    double s_ls;        /* least-squares s (eq 9 / eq 11)   */
    double s_hat;       /* s actually used                  */
    double o_raw;       /* o from eq 10 with s_hat          */
    double o_hat;       /* o actually used                  */
    double err;         /* R of eq 8                        */
} orc_fit;

/* Source pixel of S_k: output (y, x) of an n x n block reads input (sy, sx). */
static void sym_src(int k, int n, int y, int x, int *sy, int *sx)
{
    switch (k) {
    case 0: *sy = y;         *sx = x;         break; /* identity        */
    case 1: *sy = n - 1 - x; *sx = y;         break; /* rotate 90 cw    */
    case 2: *sy = n - 1 - y; *sx = n - 1 - x; break; /* rotate 180      */
    case 3: *sy = x;         *sx = n - 1 - y; break; /* rotate 270 cw   */
    case 4: *sy = y;         *sx = n - 1 - x; break; /* mirror L-R      */
    case 5: *sy = n - 1 - y; *sx = x;         break; /* mirror T-B      */
    case 6: *sy = x;         *sx = y;         break; /* transpose       */
    default: *sy = n - 1 - x; *sx = n - 1 - y; break; /* anti-transpose */
    }
}

int orc_num_domains_x(int w, const orc_params *p) { return (w - 2 * p->n) / p->t + 1; }
int orc_num_domains_y(int h, const orc_params *p) { return (h - 2 * p->n) / p->t + 1; }

/* tau: 2n x 2n domain with top-left (dy, dx) -> n x n block of 2x2 means. */
static void contract(const double *img, int w, int dy, int dx, int n, double *a)
{
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            const double *p0 = img + (size_t)(dy + 2 * y) * w + (dx + 2 * x);
            const double *p1 = p0 + w;
            a[y * n + x] = 0.25 * (p0[0] + p0[1] + p1[0] + p1[1]);
        }
}

/* B = S_k(A) for an n x n block. */
static void apply_sym(int k, int n, const double *A, double *B)
{
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            int sy, sx;
            sym_src(k, n, y, x, &sy, &sx);
            B[y * n + x] = A[sy * n + sx];
        }
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Least squares, quantisation and residual for one code block a and range b. */
static void fit_block(const double *a, const double *b, int m, const orc_params *p, orc_fit *f)
{
    double Sa = 0.0, Sb = 0.0, Saa = 0.0, Sab = 0.0;
    for (int i = 0; i < m; ++i) {
        Sa += a[i];
        Sb += b[i];
        Saa += a[i] * a[i];
        Sab += a[i] * b[i];
    }
    const double md = (double)m;
    const double den = md * Saa - Sa * Sa;                        /* domain variance */
    const double s = (den == 0.0) ? 0.0 : (md * Sab - Sa * Sb) / den; /* eq 9 / eq 11 */
    f->s_ls = s;
    if (p->s_bits > 0) {
        const double Ls = (double)((1 << (p->s_bits - 1)) - 1);
        const double sc = clampd(s, -1.0, 1.0);
        f->c = (int32_t)round(sc * Ls);
        f->s_hat = (double)f->c / Ls;
    } else {
        f->c = 0;
        f->s_hat = s;
    }
    const double o = (Sb - f->s_hat * Sa) / md;                   /* eq 10 / eq 12 */
    f->o_raw = o;
    if (p->o_bits > 0) {
        const double P = (double)((1 << p->bit_depth) - 1);
        const double Lo = (double)((1 << (p->o_bits - 1)) - 1);
        const double oc = clampd(o, -P, P);
        f->e = (int32_t)round(oc * Lo / P);
        f->o_hat = (double)f->e * P / Lo;
    } else {
        f->e = 0;
        f->o_hat = o;
    }
    double R = 0.0;                                                /* eq 8 */
    for (int i = 0; i < m; ++i) {
        const double r = f->s_hat * a[i] + f->o_hat - b[i];
        R += r * r;
    }
    f->err = R;
}

static void range_block(const double *img, int w, int r, int n, double *b)
{
    const int nx = w / n;
    const int ry = (r / nx) * n, rx = (r % nx) * n;
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) b[y * n + x] = img[(size_t)(ry + y) * w + rx + x];
}

/* Evaluate one candidate (range r, domain d, symmetry k). */
int orc_fit_candidate(const double *img, int w, int h, const orc_params *p, int r, int d, int k,
                      orc_fit *out)
{
    const int n = p->n, m = n * n;
    const int U = orc_num_domains_x(w, p);
    double *buf = (double *)malloc(sizeof(double) * 3 * (size_t)m);
    if (!buf) return -1;
    double *a0 = buf, *a = buf + m, *b = buf + 2 * m;
    (void)h;
    range_block(img, w, r, n, b);
    contract(img, w, (d / U) * p->t, (d % U) * p->t, n, a0);
    apply_sym(k, n, a0, a);
    fit_block(a, b, m, p, out);
    out->d = d;
    out->k = k;
    free(buf);
    return 0;
}

/* Exhaustive search for the listed ranges (Algorithm 2 / Algorithm 3). */
int orc_encode(const double *img, int w, int h, const orc_params *p, const int32_t *ranges,
               int n_ranges, orc_fit *out, int n_threads)
{
    const int n = p->n, m = n * n;
    const int U = orc_num_domains_x(w, p), V = orc_num_domains_y(h, p);
    int fail = 0;
    (void)n_threads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1)
    for (int ri = 0; ri < n_ranges; ++ri) {
        double *buf = (double *)malloc(sizeof(double) * 3 * (size_t)m);
        if (!buf) {
            fail = 1;
            continue;
        }
        double *a0 = buf, *a = buf + m, *b = buf + 2 * m;
        range_block(img, w, ranges[ri], n, b);
        orc_fit best;
        memset(&best, 0, sizeof best);
        best.err = INFINITY;
        for (int d = 0; d < U * V; ++d) {
            contract(img, w, (d / U) * p->t, (d % U) * p->t, n, a0);
            for (int k = 0; k < 8; ++k) {
                orc_fit f;
                apply_sym(k, n, a0, a);
                fit_block(a, b, m, p, &f);
                if (f.err < best.err) { /* strict: the first minimum is kept */
                    best = f;
                    best.d = d;
                    best.k = k;
                }
            }
        }
        out[ri] = best;
        free(buf);
    }
    return fail ? -1 : 0;
}

/* One Jacobi step of the decoder: dst = W(src) for every range. */
static void decode_step(const double *src, double *dst, int w, int h, const orc_params *p,
                        const int32_t *dom, const int32_t *sym, const double *s_hat,
                        const double *o_hat)
{
    const int n = p->n;
    const int nx = w / n, ny = h / n;
    const int U = orc_num_domains_x(w, p);
    for (int r = 0; r < nx * ny; ++r) {
        const int ry = (r / nx) * n, rx = (r % nx) * n;
        const int dy = (dom[r] / U) * p->t, dx = (dom[r] % U) * p->t;
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                int sy, sx;
                sym_src(sym[r], n, y, x, &sy, &sx);
                const double *p0 = src + (size_t)(dy + 2 * sy) * w + (dx + 2 * sx);
                const double *p1 = p0 + w;
                const double a = 0.25 * (p0[0] + p0[1] + p1[0] + p1[1]);
                dst[(size_t)(ry + y) * w + rx + x] = s_hat[r] * a + o_hat[r];
            }
    }
}

/* Decode: `iters` Jacobi steps from a flat image of value `init`.  With
 * clamp != 0 the final image is clamped to [0, P].  `trace` (optional, size
 * iters+1 images) receives every iterate before clamping. */
int orc_decode(int w, int h, const orc_params *p, const int32_t *dom, const int32_t *sym,
               const double *s_hat, const double *o_hat, int iters, double init, int clamp,
               double *out, double *trace)
{
    const size_t npx = (size_t)w * h;
    double *x0 = (double *)malloc(sizeof(double) * npx);
    double *x1 = (double *)malloc(sizeof(double) * npx);
    if (!x0 || !x1) {
        free(x0);
        free(x1);
        return -1;
    }
    for (size_t i = 0; i < npx; ++i) x0[i] = init;
    if (trace) memcpy(trace, x0, sizeof(double) * npx);
    for (int it = 0; it < iters; ++it) {
        decode_step(x0, x1, w, h, p, dom, sym, s_hat, o_hat);
        double *tmp = x0;
        x0 = x1;
        x1 = tmp;
        if (trace) memcpy(trace + (size_t)(it + 1) * npx, x0, sizeof(double) * npx);
    }
    const double P = (double)((1 << p->bit_depth) - 1);
    for (size_t i = 0; i < npx; ++i) out[i] = clamp ? clampd(x0[i], 0.0, P) : x0[i];
    free(x0);
    free(x1);
    return 0;
}

/* Differentiable refinement (the decoder with real-valued s and o):
 * loss L = (1/N) sum_p (x_T[p] - ref[p])^2 of the unrolled, unclamped decode
 * x_{t+1} = W(x_t) from x_0 = init (W: every range's pixels set to
 * s_r * S_k(tau(x_t restricted to its domain)) + o_r, as in decode_step), and
 * its gradient with respect to every s_r and o_r by the adjoint of the
 * iteration, taken step by step in reverse:
 *   g_T = 2 (x_T - ref) / N;
 *   for t = T-1 .. 0:  with a_t[p] the contracted, transformed domain value
 *   that output pixel p of range r reads from x_t,
 *     dL/ds_r += sum_{p in r} g_{t+1}[p] a_t[p],   dL/do_r += sum_{p in r} g_{t+1}[p],
 *     g_t = W'^T g_{t+1}: each output pixel p adds s_r/4 g_{t+1}[p] to each of
 *     the four source pixels it averages.
 * Every iterate is kept (plain, no checkpointing). */
int orc_refine_grad(int w, int h, const orc_params *p, const int32_t *dom, const int32_t *sym, const double *s,
                    const double *o, int iters, double init, const double *ref, double *loss, double *grad_s,
                    double *grad_o)
{
    const size_t npx = (size_t)w * h;
    const int n = p->n, nx = w / n, ny = h / n, R = nx * ny;
    const int U = orc_num_domains_x(w, p);
    double *x = (double *)malloc(sizeof(double) * npx * (size_t)(iters + 1));
    double *g = (double *)malloc(sizeof(double) * npx);
    double *g2 = (double *)malloc(sizeof(double) * npx);
    if (!x || !g || !g2) {
        free(x);
        free(g);
        free(g2);
        return -1;
    }
    for (size_t i = 0; i < npx; ++i) x[i] = init;
    for (int t = 0; t < iters; ++t) decode_step(x + npx * t, x + npx * (t + 1), w, h, p, dom, sym, s, o);
    const double *xT = x + npx * iters;
    double se = 0.0;
    for (size_t i = 0; i < npx; ++i) {
        const double dlt = xT[i] - ref[i];
        se += dlt * dlt;
        g[i] = 2.0 * dlt / (double)npx;
    }
    *loss = se / (double)npx;
    for (int r = 0; r < R; ++r) grad_s[r] = grad_o[r] = 0.0;
    for (int t = iters - 1; t >= 0; --t) {
        const double *xt = x + npx * t;
        for (size_t i = 0; i < npx; ++i) g2[i] = 0.0;
        for (int r = 0; r < R; ++r) {
            const int ry = (r / nx) * n, rx = (r % nx) * n;
            const int dy = (dom[r] / U) * p->t, dx = (dom[r] % U) * p->t;
            for (int y = 0; y < n; ++y)
                for (int xx = 0; xx < n; ++xx) {
                    int sy, sx;
                    sym_src(sym[r], n, y, xx, &sy, &sx);
                    const size_t q = (size_t)(dy + 2 * sy) * w + (dx + 2 * sx);
                    const double a = 0.25 * (xt[q] + xt[q + 1] + xt[q + w] + xt[q + w + 1]);
                    const double gp = g[(size_t)(ry + y) * w + rx + xx];
                    grad_s[r] += gp * a;
                    grad_o[r] += gp;
                    const double back = 0.25 * s[r] * gp;
                    g2[q] += back;
                    g2[q + 1] += back;
                    g2[q + w] += back;
                    g2[q + w + 1] += back;
                }
        }
        double *tmp = g;
        g = g2;
        g2 = tmp;
    }
    (void)ny;
    free(x);
    free(g);
    free(g2);
    return 0;
}

/* Peak signal-to-noise ratio 10*log10(P^2 / MSE) in dB. */
double orc_psnr(const double *ref, const double *img, size_t npx, int bit_depth)
{
    const double P = (double)((1 << bit_depth) - 1);
    double se = 0.0;
    for (size_t i = 0; i < npx; ++i) {
        const double dlt = ref[i] - img[i];
        se += dlt * dlt;
    }
    const double mse = se / (double)npx;
    return mse == 0.0 ? INFINITY : 10.0 * log10(P * P / mse);
}
