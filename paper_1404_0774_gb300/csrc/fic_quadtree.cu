// Adaptive quadtree: the split decision between levels and the gather of the
// kept leaves (the per-level search is the encode pipeline itself).
#include <algorithm>

#include "fic_internal.cuh"

namespace fic {

// Level with range size n (nx ranges per row): every active range whose best
// map has collage RMS error sqrt(E/m) > rms_split is split into its four
// quadrants (marked active at the next level, which the caller zeroed);
// the others are leaves.  The last level keeps every active range.
__global__ void k_qt_split(int R, int nx, int m, const fic_map *maps, const int *active, double rms_split, int last,
                           int *leaf, int *active_next)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    if (!active[r]) {
        leaf[r] = 0;
        return;
    }
    const bool split = !last && sqrt(maps[r].err / (double)m) > rms_split;
    leaf[r] = split ? 0 : 1;
    if (split) {
        const int ry = r / nx, rx = r - (r / nx) * nx, nx2 = 2 * nx;
        active_next[(2 * ry) * nx2 + 2 * rx] = 1;
        active_next[(2 * ry) * nx2 + 2 * rx + 1] = 1;
        active_next[(2 * ry + 1) * nx2 + 2 * rx] = 1;
        active_next[(2 * ry + 1) * nx2 + 2 * rx + 1] = 1;
    }
}

// Block l: stable compaction of level l's leaf flags (range indices in
// order into list[l]) with warp ballots, 1024 flags a round; counts[1 + l] =
// leaves of level l, counts[1 + kMaxLevels + l] = active ranges of level l.
__global__ void __launch_bounds__(1024) k_qt_leaves(QtLevels lv, int *lists, int *counts)
{
    __shared__ int wsum[32];
    __shared__ int base_s, nact_s;
    const int l = blockIdx.x;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int R = lv.R[l];
    const int *leaf = lv.leaf[l];
    const int *active = lv.active[l];
    int *list = lists + lv.list_off[l];
    if (t == 0) {
        base_s = 0;
        nact_s = 0;
    }
    __syncthreads();
    int nact = 0;
    for (int i0 = 0; i0 < R; i0 += 1024) {
        const int r = i0 + t;
        const bool f = r < R && leaf[r] != 0;
        if (r < R && active[r]) ++nact;
        const unsigned b = __ballot_sync(0xffffffffu, f);
        if (lane == 0) wsum[w] = __popc(b);
        __syncthreads();
        if (w == 0) {
            const int v = wsum[lane];
            int x = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            wsum[lane] = x - v;
        }
        __syncthreads();
        const int base = base_s, wbase = wsum[w];
        if (f) list[base + wbase + __popc(b & ((1u << lane) - 1u))] = r;
        __syncthreads();
        if (t == 1023) base_s = base + wbase + __popc(b);
    }
    atomicAdd(&nact_s, nact);
    __syncthreads();
    if (t == 0) {
        counts[1 + l] = base_s;
        counts[1 + kMaxLevels + l] = nact_s;
    }
}

// Every leaf, in order (level, then range index): leaf i of level l goes to
// the sum of the earlier levels' counts plus i.  counts[0] = leaves in all,
// counts[1 + 2 kMaxLevels] = 1 if a leaf carries FIC_MAP_ERROR (zeroed by the
// caller).
__global__ void k_qt_write(QtLevels lv, const int *lists, int *counts, fic_qmap *out, int cap)
{
    int base = 0;
    for (int l = 0; l < lv.levels; ++l) {
        const int nl = counts[1 + l];
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += gridDim.x * blockDim.x) {
            const int pos = base + i;
            if (pos >= cap) break;
            const int r = lists[lv.list_off[l] + i];
            const int nx = lv.nx[l], n = lv.n[l];
            fic_qmap q;
            q.x = (uint32_t)((r % nx) * n);
            q.y = (uint32_t)((r / nx) * n);
            q.size = (uint32_t)n;
            q.level = (uint32_t)l;
            q.map = lv.maps[l][r];
            out[pos] = q;
            if (q.map.info & FIC_MAP_ERROR) counts[1 + 2 * kMaxLevels] = 1;
        }
        base += nl;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) counts[0] = base;
}

cudaError_t launch_qt_split(int R, int nx, int m, const fic_map *maps, const int *active, double rms_split, int last,
                            int *leaf, int *active_next, cudaStream_t st)
{
    k_qt_split<<<(R + 255) / 256, 256, 0, st>>>(R, nx, m, maps, active, rms_split, last, leaf, active_next);
    return cudaGetLastError();
}

cudaError_t launch_qt_gather(const QtLevels &lv, int *lists, fic_qmap *out, int cap, int *counts, cudaStream_t st)
{
    k_qt_leaves<<<lv.levels, 1024, 0, st>>>(lv, lists, counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_qt_write<<<std::max(1, std::min(1024, (cap + 255) / 256)), 256, 0, st>>>(lv, lists, counts, out, cap);
    return cudaGetLastError();
}

}  // namespace fic
