/*
 * fic.h -- C ABI of the GB300 PIFS fractal-encoding library (libfic.so).
 *
 * The library implements the hot path of partitioned-iterated-function-system
 * (PIFS) fractal image encoding after Haque et al., "GPU Accelerated Fractal
 * Image Compression for Medical Imaging in Parallel Computing Platform"
 * (arXiv 1404.0774): the exhaustive range-domain search of Section V
 * (Algorithm 2, parallelised per range as in Algorithm 3), and the decoder
 * that iterates the resulting maps (the "decoding" of the abstract and
 * Section VI).  Everything runs on one CUDA GPU; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Image: row-major, `pitch_px` elements per row (pitch_px >= w).  Pixel type
 *    is uint8_t when bit_depth <= 8 and uint16_t when 8 < bit_depth <= 12;
 *    values must lie in [0, 2^bit_depth - 1].
 *  - Ranges (Section V, Section VI): non-overlapping n x n blocks; range
 *    r = j*(w/n) + i has its top-left pixel at row n*j, column n*i.
 *  - Domains (Section V, Algorithm 1): 2n x 2n blocks on a grid of spacing t
 *    (the paper's STEP); domain d = v*U + u, U = (w-2n)/t + 1, has its top-left
 *    pixel at row t*v, column t*u.  They are contracted by the 2x2 mean.
 *  - Symmetries (Section V: rotations and mirroring), k = 0..7: identity,
 *    rotate 90 cw, rotate 180, rotate 270 cw, mirror left-right, mirror
 *    top-bottom, transpose, anti-transpose.  Output pixel (y, x) of S_k(A)
 *    reads A at (y,x), (n-1-x,y), (n-1-y,n-1-x), (x,n-1-y), (y,n-1-x),
 *    (n-1-y,x), (x,y), (n-1-x,n-1-y) respectively.
 *  - Candidate index = 8*d + k; the search order is d-major, k-minor and the
 *    first of equal minima wins (Algorithm 2, strict comparison).
 *  - Contrast s by least squares (eq 9, with the domain-variance denominator
 *    n*sum(a^2) - (sum a)^2 stated after eq 10; s = 0 for a flat domain,
 *    eq 11), clamped to [-1, 1] and rounded half away from zero to c/Ls,
 *    Ls = 2^(s_bits-1) - 1.  Brightness o = (sum b - s_hat*sum a)/m (eq 10
 *    with the quantised s), clamped to [-P, P], P = 2^bit_depth - 1, rounded
 *    half away from zero to e*P/Lo, Lo = 2^(o_bits-1) - 1.  Collage error
 *    R = sum (s_hat*a_i + o_hat - b_i)^2 (eq 8).
 *  - Pointers may be host or device memory; the library detects which
 *    (cudaPointerGetAttributes) and moves host data itself: fic_encode reads a
 *    page-locked host image with a copy kernel (16-byte aligned, rows
 *    contiguous; otherwise, and for pageable memory, by a copy-engine
 *    transfer) and its map output kernel writes page-locked host maps in
 *    place (pageable maps are copied back).  The caller owns every buffer.
 *    `stream` is a cudaStream_t (NULL = legacy default stream).  Calls on one
 *    stream are ordered; the host-pointer variants synchronise the stream
 *    before returning.
 *  - Errors: every call returns FIC_OK (0) or a negative FIC_ERR_* code and
 *    never aborts; fic_status_str() gives a message.
 */
#ifndef FIC_H
#define FIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FIC_OK = 0,
    FIC_ERR_BAD_ARG = -1,   /* null pointer, bad parameter value              */
    FIC_ERR_SIZE = -2,      /* w/h not multiples of n, smaller than 2n, ...  */
    FIC_ERR_BITDEPTH = -3,  /* bit_depth outside 1..12, bad s_bits/o_bits     */
    FIC_ERR_CAPACITY = -4,  /* output or workspace buffer too small           */
    FIC_ERR_CUDA = -5,      /* a CUDA runtime call failed                     */
    FIC_ERR_TIMEOUT = -6,   /* a bounded device-side wait ran out             */
    FIC_ERR_UNSUPPORTED = -7 /* valid parameters this library does not handle */
};

/* Search implementation. */
enum {
    FIC_SEARCH_AUTO = 0, /* the tensor-core search (every range size n)       */
    FIC_SEARCH_TC = 1,   /* FP16 tcgen05 tensor-core cross term + FP32 epilogue */
    FIC_SEARCH_SIMT = 2  /* plain FP32 CUDA-core search (the speedup baseline) */
};

typedef struct {
    int32_t range_size;    /* n: 4, 8 or 16                                   */
    int32_t domain_stride; /* t >= 1 (the paper's STEP)                       */
    int32_t bit_depth;     /* B: 1..12                                        */
    int32_t s_bits;        /* contrast code bits, 2..8 (5 in the workloads)   */
    int32_t o_bits;        /* brightness code bits, 2..10 (7)                 */
    int32_t decode_iters;  /* Jacobi iterations of fic_decode (10)            */
    int32_t search;        /* FIC_SEARCH_*                                    */
    int32_t n_split;       /* candidate-dimension splits, 0 = automatic       */
    uint32_t flags;        /* FIC_FLAG_* bits                                 */
} fic_params;

/* fic_params.flags: record CUDA events around each encode phase on the
 * caller's stream (read them back with fic_last_encode_phase_ms). */
#define FIC_FLAG_PHASE_TIMING 0x1u
/* fic_params.flags: screen every range and every domain.  By default the
 * search skips what Section V says needs no search: shadow (constant) ranges,
 * and flat (zero-variance) domains, whose candidates all share one residual
 * per range and are represented by the first of them.  The maps are the same
 * either way; this flag exists to measure and test the dense search. */
#define FIC_FLAG_DENSE 0x2u
/* fic_params.flags: resolve every screened range by the exact exhaustive
 * scan (integer cross terms and exact code decisions over all 8*D
 * candidates) instead of certifying the screened lists.  The maps are the
 * same, each flagged FIC_MAP_FALLBACK; this flag exists to test that scan and
 * to time it. */
#define FIC_FLAG_EXACT_SCAN 0x4u

/* One map per range: range -> (domain, symmetry, s, o) and its collage error. */
typedef struct {
    uint32_t range_idx;  /* r                                                 */
    uint32_t domain_idx; /* d                                                 */
    int32_t iso;         /* k in 0..7                                         */
    int32_t s_code;      /* c in [-Ls, Ls]; s_hat = c / Ls                    */
    int32_t o_code;      /* e in [-Lo, Lo]; o_hat = e * P / Lo                */
    float s;             /* s_hat                                             */
    float o;             /* o_hat                                             */
    uint32_t info;       /* FIC_MAP_* bits                                    */
    double err;          /* eq 8 residual: exact value rounded to FP64        */
} fic_map;

#define FIC_MAP_FALLBACK 0x1u /* resolved by the exact full rescan           */
#define FIC_MAP_ERROR 0x2u    /* a bounded device wait timed out: invalid    */

/* Fill `p` with the defaults of the workloads (n=8, t=8, B=8, 5/7 bits,
 * 10 decode iterations, automatic search). */
void fic_default_params(fic_params *p);

/* Number of ranges and domains of a w x h image under `p`; returns FIC_OK or
 * an error for invalid sizes.  Either output pointer may be NULL. */
int fic_counts(int w, int h, const fic_params *p, int64_t *n_ranges, int64_t *n_domains);

/* Device workspace bytes that fic_encode needs for a w x h image. */
int fic_encode_workspace_size(int w, int h, const fic_params *p, size_t *bytes);

/*
 * fic_encode -- exhaustive range-domain search (Section V, Algorithms 1-3).
 *   img        w x h image (pitch_px elements per row), host or device.
 *   maps       output, one fic_map per range in range order (host or device);
 *              maps_cap >= number of ranges.
 *   n_maps     output (host), number of maps written; may be NULL.
 *   workspace  device buffer of at least fic_encode_workspace_size() bytes,
 *              256-byte aligned (FIC_ERR_BAD_ARG otherwise; cudaMalloc and
 *              torch allocations are), or NULL to let the library allocate
 *              (cudaMallocAsync) and free it on `stream`.
 * Every map is the exact minimiser of eq 8 over all 8*D candidates with the
 * lowest-index tie-break; codes are decided in FP64 as described above.
 */
int fic_encode(const void *img, int w, int h, int pitch_px, const fic_params *p, fic_map *maps,
               int maps_cap, int *n_maps, void *workspace, size_t workspace_bytes, void *stream);

/*
 * fic_decode -- iterate the maps (decoding, abstract and Section VI).
 *   Starts from a flat image of value `init`, applies p->decode_iters Jacobi
 *   steps x <- s_hat * S_k(tau(x[domain])) + o_hat over all ranges (FP32, no
 *   clamping inside the iteration), then clamps to [0, P] into `out`
 *   (w*h floats, row-major, host or device).  `maps` (n_maps = number of
 *   ranges, host or device) is read-only; host maps are validated (domain and
 *   symmetry in range), device maps must come from fic_encode with the same
 *   w, h and parameters.  `workspace` as in fic_encode, of
 *   fic_decode_workspace_size() bytes (NULL = allocate).
 */
int fic_decode(const fic_map *maps, int n_maps, int w, int h, const fic_params *p, float init,
               float *out, void *workspace, size_t workspace_bytes, void *stream);

/* Device workspace bytes that fic_decode needs for a w x h image. */
int fic_decode_workspace_size(int w, int h, const fic_params *p, size_t *bytes);

/*
 * fic_decode_scaled -- resolution-independent decoding (the property the
 *   paper's introduction credits fractal coding with): the maps of a w x h
 *   encode decoded at 2^scale_log2 times that size.  Every range block and
 *   domain position and side is scaled (range n*z at (x*z, y*z), domain 2n*z
 *   at (u*t*z, v*t*z), z = 2^scale_log2) while the 2x2 contraction, the
 *   symmetries and s, o stay as encoded; iterated as fic_decode does.
 *   scale_log2 in [-3, 3]; for z < 1 the range side n, the domain stride t,
 *   w and h must be multiples of 1/z.  out: (w*z) x (h*z) floats.  At z = 1
 *   this is fic_decode.  Averaging 2x2 blocks of the unclamped decode at 2z
 *   gives the unclamped decode at z (the contraction commutes with the
 *   symmetries), so every scale decodes one consistent image.
 */
int fic_decode_scaled(const fic_map *maps, int n_maps, int w, int h, const fic_params *p, int scale_log2, float init,
                      float *out, void *workspace, size_t workspace_bytes, void *stream);
int fic_decode_scaled_workspace_size(int w, int h, const fic_params *p, int scale_log2, size_t *bytes);

/* Human-readable message for a status code. */
const char *fic_status_str(int status);

/* Counters of the last fic_encode on this host thread (diagnostics):
 * out[0] = ranges resolved by the exact full rescan, out[1] = number of
 * candidate lists, out[2] = search implementation used (FIC_SEARCH_*). */
int fic_last_encode_stats(int64_t out[4]);

/*
 * fic_cross_terms -- the contraction alone, for testing: runs the encode's
 *   prep and the selected search path's cross-term stage and writes
 *   Xt[r][c] = sum_i q'_i b'_i - e_r f_d / m = (m*X - Sq*Sb)/m as FP32 for
 *   every range r and candidate c (row-major, R x 8D floats, DEVICE memory
 *   `out`), where X = sum_i q_i b_i is the eq 9 cross term (q the 2x2 sums of
 *   S_k(domain d), b the range pixels), Sq = sum q, Sb = sum b.  `img` as in
 *   fic_encode (device); workspace as fic_encode (NULL = allocate).
 *   Returns FIC_ERR_TIMEOUT if a bounded device wait expired.
 */
int fic_cross_terms(const void *img, int w, int h, int pitch_px, const fic_params *p, float *out,
                    void *workspace, size_t workspace_bytes, void *stream);

/*
 * fic_encode_static -- fic_encode for callers that may not allocate device
 *   memory (no counterpart in the paper: this is a deployment aid).
 *
 *   Some hosts forbid device allocation by a library: a plug-in whose host
 *   application owns all GPU memory, a real-time pipeline that reserves every
 *   buffer at start-up, a process under a device-memory cap it does not
 *   control.  This call allocates nothing (no cudaMalloc, cudaFree or other
 *   allocating routine): its scratch is a static device array of
 *   FIC_STATIC_SCRATCH_BYTES that each GPU loading the library keeps until
 *   the process exits.  The caller still passes the image and the maps
 *   buffer (host or device, as for fic_encode).
 *
 *   - Images whose workspace (fic_encode_workspace_size) exceeds
 *     FIC_STATIC_SCRATCH_BYTES are rejected with FIC_ERR_CAPACITY before any
 *     device work; e.g. 256x256 with 8x8 ranges fits, 512x512 at stride 4
 *     does not.
 *   - The first call on each device looks up the array's device address (and
 *     may load the array onto that device); make that first call before any
 *     stream capture on that device.  The address is kept per device and
 *     context: after the device's context is destroyed and created again
 *     (cudaDeviceReset), the next call looks it up anew, so that call too
 *     belongs outside a capture.
 *   - Every call on a device shares the one array, which keeps the previous
 *     call's contents (each call initialises what it needs).  Calls whose
 *     work overlaps on the GPU -- concurrent streams, or several host threads
 *     -- race on it: serialise them.
 *   - FIC_FLAG_PHASE_TIMING is rejected (it would create CUDA events).
 */
#define FIC_STATIC_SCRATCH_BYTES (32u << 20)
int fic_encode_static(const void *img, int w, int h, int pitch_px, const fic_params *p, fic_map *maps,
                      int maps_cap, int *n_maps, void *stream);

/* One leaf of an adaptive quadtree encode (fic_encode_quadtree). */
typedef struct {
    uint32_t x, y;   /* top-left pixel of the range block                       */
    uint32_t size;   /* its side n = range_size >> level                        */
    uint32_t level;  /* 0 = the largest blocks                                  */
    fic_map map;     /* its map; range_idx and domain_idx index the grids of its
                        level: w/n ranges per row, domains 2n x 2n at stride n
                        with (w-2n)/n + 1 per row                               */
} fic_qmap;          /* 56 bytes */

/*
 * fic_encode_quadtree -- adaptive quadtree encode.  The paper searches one
 *   range size; this applies the same exhaustive search (Section V, eq 8-12,
 *   same quantisation, tie-break and exactness as fic_encode) at several:
 *   level 0 tiles the image with p->range_size ranges; a range whose best map
 *   has collage RMS error sqrt(E/m) > rms_split (compared in FP64) is
 *   replaced by its four quadrants at the next level, down to min_size, whose
 *   ranges are always kept.  At a level with range size n the domains are
 *   2n x 2n at stride n (p->domain_stride is ignored).  Each level is one
 *   encode over that level's active ranges only.
 *   maps       output leaves (host or device) ordered by level, then by range
 *              index within the level; maps_cap >= (w/min_size)*(h/min_size).
 *   n_maps     output (host): number of leaves.  The call waits for `stream`.
 *   workspace  device buffer of fic_quadtree_workspace_size() bytes, 256-byte
 *              aligned, or NULL to allocate on `stream`.
 *   Launch shapes: with p->search == FIC_SEARCH_AUTO and p->n_split == 0 each
 *   level's search kernel (tensor-core where supported, else FP32) and the
 *   number of CTAs its candidate dimension is spread over are chosen by
 *   timing the candidates once per geometry and caching the fastest (the
 *   maps do not depend on the choice); otherwise p->search / p->n_split fix
 *   them.
 *   Sizes: range_size 16 or 8, min_size 4, 8 or 16 with min_size <=
 *   range_size; w and h multiples of range_size, at least 2*range_size.
 *   FIC_FLAG_PHASE_TIMING: record events around each level's search (read
 *   them with fic_last_quadtree_phase_ms).
 */
int fic_encode_quadtree(const void *img, int w, int h, int pitch_px, const fic_params *p, int min_size,
                        float rms_split, fic_qmap *maps, int maps_cap, int *n_maps, void *workspace,
                        size_t workspace_bytes, void *stream);
int fic_quadtree_workspace_size(int w, int h, const fic_params *p, int min_size, size_t *bytes);

/* Per level of the last fic_encode_quadtree on this host thread: out[0] =
 * number of levels L, then for level l at out[1 + 4l ..]: search kernel used
 * (FIC_SEARCH_*), CTA target of its candidate split (waves x SMs), ranges
 * screened (active), leaves kept. */
int fic_last_quadtree_stats(int64_t out[17]);

/* Search time (ms) of each level of the last fic_encode_quadtree on this host
 * thread that ran with FIC_FLAG_PHASE_TIMING: out[l] for level l (0 past the
 * last level).  Waits for those events; FIC_ERR_BAD_ARG if there are none. */
int fic_last_quadtree_phase_ms(double out[3]);

/* One slice of a batch (fic_encode_batch); every pointer is device memory. */
typedef struct {
    const void *img;   /* w x h image, row pitch pitch_px elements; uint8 for
                          bit_depth <= 8, else uint16                          */
    int32_t w, h, pitch_px;
    fic_map *maps;     /* output: one map per range of this slice (in range
                          order), (w/n)*(h/n) of them                          */
} fic_slice;

/*
 * fic_encode_batch -- encode n slices (1 <= n <= 1024) of possibly different
 *   sizes with the same parameters: for each slice exactly what fic_encode
 *   computes.  The slices, sorted by size, are dealt round-robin to six parts
 *   that run as concurrent pipelines; in each, every stage of the encode is one
 *   launch over its slices (the slice is the last grid dimension), and the
 *   search is one persistent kernel that walks a queue of (slice, candidate
 *   split, range tile) work items.  The launches form one CUDA graph, captured on the first
 *   call for a batch (which also runs it) and replayed while the slice table,
 *   parameters and workspace stay the same (a different batch captures a new
 *   graph; one graph is kept per host thread).
 *   workspace  device, fic_batch_workspace_size() bytes, 256-byte aligned
 *              (required: the graph refers to it; it also holds the slice
 *              table the kernels read, written by the first call).
 *   Asynchronous on `stream` (the first call for a batch waits for its
 *   stream once, after writing the slice table); the maps are ready when the
 *   stream is.  Bounded device waits that expire flag the affected maps
 *   FIC_MAP_ERROR.  FIC_FLAG_PHASE_TIMING is rejected; more than 1024 slices:
 *   FIC_ERR_CAPACITY.
 */
int fic_encode_batch(const fic_slice *slices, int n, const fic_params *p, void *workspace, size_t workspace_bytes,
                     void *stream);
int fic_batch_workspace_size(const fic_slice *slices, int n, const fic_params *p, size_t *bytes);

/* Completion time (ms) of each slice of the last graph replay of
 * fic_encode_batch on this host thread (the first call for a batch runs
 * eagerly and records none), from the start of the batch: events recorded
 * inside the graph; waits for them.  Every stage covers every slice, so all
 * slices complete with the batch: each entry is the batch's time.  out has n
 * entries. */
int fic_last_batch_slice_ms(float *out, int n);

/*
 * Differentiable refinement (fic_refine*): the decoder with real-valued FP32
 * contrast s_r and offset o_r per range (each map's domain and symmetry
 * fixed), unrolled for `iters` Jacobi iterations without clamping from a flat
 * x_0 = init:  x_{t+1}[p] = s_r * a_t[p] + o_r, where a_t[p] is the 2x2 mean
 * of x_t that S_k places at pixel p of range r (the maps of eq 6, iterated as
 * the decoder does).  The adjoint of that iteration gives dL/ds and dL/do for
 * a loss L of x_T.  The paper decodes with the fitted coefficients; refining
 * them against the decoded image rather than the collage bound is an
 * extension of it.  Every pointer is device memory; maps as fic_encode wrote
 * them for this w, h and parameters.  Iterates are checkpointed every second
 * step: ckpt holds ceil(iters/2) w x h float images (x_0, x_2, ...), and the
 * odd ones are recomputed in the reverse sweep.  The adjoint sums in a fixed
 * order (no atomics): results are deterministic.
 */
int fic_refine_workspace_size(int w, int h, const fic_params *p, int iters, size_t *bytes);
/* x_out = x_T (w x h floats); ckpt as above (filled for fic_refine_backward). */
int fic_refine_forward(const fic_map *maps, int w, int h, const fic_params *p, const float *s, const float *o,
                       float init, int iters, float *x_out, float *ckpt, void *workspace, size_t workspace_bytes,
                       void *stream);
/* grad_x = dL/dx_T (w x h); writes dL/ds and dL/do (one per range). */
int fic_refine_backward(const fic_map *maps, int w, int h, const fic_params *p, const float *s, const float *o,
                        int iters, const float *ckpt, const float *grad_x, float *grad_s, float *grad_o,
                        void *workspace, size_t workspace_bytes, void *stream);
/* fic_refine -- the whole refinement: Adam (beta1 0.9, beta2 0.999, eps 1e-8,
 * step size lr on s and on o/P) for `steps` steps on L = mean((x_T - img)^2),
 * x_0 = 2^(B-1).  s and o (one per range) are read and updated in place.
 * loss (optional, steps + 1 floats): L before each step and after the last.
 * img as in fic_encode but device memory.  One step is a CUDA graph replay;
 * asynchronous on `stream`. */
int fic_refine(const void *img, int w, int h, int pitch_px, const fic_params *p, const fic_map *maps, float *s,
               float *o, int steps, int iters, float lr, float *loss, void *workspace, size_t workspace_bytes,
               void *stream);

/*
 * fic_set_wait_limit_ns -- wall-clock limit of each bounded device-side wait
 *   of the tensor-core search (an mbarrier wait for a shared-memory stage, a
 *   TMEM accumulator or a work item; measured with %globaltimer).  When a
 *   wait runs out, the CTA records the error, stops, waits (up to 2 s) for the
 *   copies and MMAs it has already issued, frees its TMEM and exits; the
 *   affected maps carry FIC_MAP_ERROR and the synchronous calls return
 *   FIC_ERR_TIMEOUT.  The GPU context stays usable.  ns = 0 restores the
 *   default of 2e9 (2 s).  Process-wide; applies to launches made after the
 *   call (a batch graph captured earlier keeps the limit it was captured
 *   with).  Always returns FIC_OK.  The paper has no counterpart: this
 *   lets a caller bound how long a stuck search may hold the GPU, and lets
 *   tests drive the timeout path without any fault.
 */
int fic_set_wait_limit_ns(uint64_t ns);
uint64_t fic_get_wait_limit_ns(void);

/* Phase durations (ms) of the last fic_encode on this host thread that ran
 * with FIC_FLAG_PHASE_TIMING: out[0] prep, out[1] search, out[2] re-score,
 * out[3] exact fallback scans and map output (one launch), out[4] 0 (kept
 * so that the array layout is unchanged).  Waits for those events. */
int fic_last_encode_phase_ms(double out[5]);

#ifdef __cplusplus
}
#endif
#endif /* FIC_H */
