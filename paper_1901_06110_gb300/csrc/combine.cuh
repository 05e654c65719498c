// Combine step of the TMA stencil: each tile and offset slice of phase 1 leaves
// a partial region (the tile plus the halo its mirrored terms reach); a pixel's
// sum is the fixed-order sum of the regions that cover it.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace dsg {

constexpr int kTmaTH = 16;   // tile rows of phase 1
constexpr int kTmaTW = 128;  // tile columns of phase 1

// Sum of the partial regions covering pixel (i, j), in a fixed order.  The region
// of tile (ty, tx) spans rows ty*kTmaTH .. ty*kTmaTH + kTmaTH + rs - 1 and columns
// tx*kTmaTW - rs .. tx*kTmaTW + kTmaTW + rs - 1, so with rs <= kTmaTH only the own tile row
// and the one above, and the own tile column and its two neighbours, can cover it.
__device__ __forceinline__ float gather_partials(const Cover& cv, int i, int j) {
    const int rs = cv.rs;
    const int RW = kTmaTW + 2 * rs;
    const size_t region = (size_t)(kTmaTH + rs) * RW;
    const int ty = i / kTmaTH, tx = j / kTmaTW;
    const int li = i - ty * kTmaTH, lj = j - tx * kTmaTW;
    const bool up = ty >= 1 && li < rs;
    const bool left = tx >= 1 && lj < rs;
    const bool right = tx + 1 < cv.tiles_x && lj >= kTmaTW - rs;
    // (tile, cell) offsets of the six candidates, upper row first, left to right
    const size_t row_up = (size_t)(ty - 1) * cv.tiles_x, row_own = (size_t)ty * cv.tiles_x;
    const size_t cell_up = (size_t)(li + kTmaTH) * RW, cell_own = (size_t)li * RW;
    size_t off[6];
    bool use[6];
    off[0] = (row_up + tx - 1) * region + cell_up + lj + kTmaTW + rs; use[0] = up && left;
    off[1] = (row_up + tx) * region + cell_up + lj + rs;           use[1] = up;
    off[2] = (row_up + tx + 1) * region + cell_up + lj - kTmaTW + rs; use[2] = up && right;
    off[3] = (row_own + tx - 1) * region + cell_own + lj + kTmaTW + rs; use[3] = left;
    off[4] = (row_own + tx) * region + cell_own + lj + rs;           use[4] = true;
    off[5] = (row_own + tx + 1) * region + cell_own + lj - kTmaTW + rs; use[5] = right;
    // unused candidates point at the own cell, so every address formed is in bounds
#pragma unroll
    for (int c = 0; c < 6; ++c)
        if (!use[c]) off[c] = off[4];
    const size_t slice_stride = (size_t)cv.tiles_y * cv.tiles_x * region;
    CompSum acc;
    const float* base = cv.part;
    for (int sl = 0; sl < cv.slices; ++sl, base += slice_stride) {
        float v[6];
#pragma unroll
        for (int c = 0; c < 6; ++c)
            v[c] = (use[c] && DSG_IN_RANGE(sl * slice_stride + off[c], cv.cap, kChkPartials)) ? __ldcg(base + off[c])
                                                                                                 : 0.f;
#pragma unroll
        for (int c = 0; c < 6; ++c)
            if (use[c]) acc.add(v[c]);
    }
    return acc.value();
}

}  // namespace dsg
