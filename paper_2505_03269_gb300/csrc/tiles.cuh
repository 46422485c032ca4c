// tiles.cuh — the persistent kernels' tile scheduler: a linear tile index
// t -> (batch, m-tile, n-tile).  Every CTA walks t = blockIdx.x,
// blockIdx.x + gridDim.x, ... so all roles of a CTA see the same sequence.
//
// Uniform batches: t enumerates batch-major tiles; within a batch either
// n-tiles (raster 0) or m-tiles (raster 1) run fastest.  Uneven batches
// (per-batch beam counts, Sec. V-B's channels with different beam sets):
// `prefix[b]` holds the number of m-tiles (of 128 rows) before batch b
// (prefix[B] = all m-tiles), so batch b starts at tile prefix[b] * n_tiles,
// and t is located by binary search.
#pragma once
#include <cstdint>

namespace tcbf {
namespace dev {

struct TileMap {
    const int *prefix;   // device [batch + 1] m-tile prefix, or nullptr for uniform batches
    int batch;
    int m_tiles;         // uniform: m-tiles per batch
    int n_tiles;
    int raster;          // 0: n fastest, 1: m fastest
};

__device__ __forceinline__ void tile_decode(const TileMap &tm, int t, int &b, int &mt, int &nt) {
    int local;
    int mtiles = tm.m_tiles;
    if (tm.prefix == nullptr) {
        const int per_b = tm.m_tiles * tm.n_tiles;
        b = t / per_b;
        local = t - b * per_b;
    } else {
        const int mt_global = t / tm.n_tiles;   // m-tile index over all batches
        int lo = 0, hi = tm.batch;              // invariant: prefix[lo] <= mt_global < prefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(tm.prefix + mid) <= mt_global) lo = mid; else hi = mid;
        }
        b = lo;
        const int base = __ldg(tm.prefix + lo);
        mtiles = __ldg(tm.prefix + lo + 1) - base;
        local = t - base * tm.n_tiles;
    }
    if (tm.raster == 0) {
        nt = local % tm.n_tiles;
        mt = local / tm.n_tiles;
    } else {
        mt = local % mtiles;
        nt = local / mtiles;
    }
}

}  // namespace dev
}  // namespace tcbf
