// Staged rows in 16-word regions, shared by the row-FIR region kernel
// (k_rowregion.cu) and the row-pass backward (k_sepbwd.cu).
//
// A thread owns the 16-word "home" region h0 .. h0 + 15 of a staged row (h0 a
// multiple of 16) and reads its window as 16-byte units from h0 on.  Rows are
// staged swizzled by 16-byte units: unit f lives at unit
// (f & ~3) | ((f & 3) ^ ((f >> 3) & 3)), so the 8 lanes of a quarter-warp
// that read unit v of 8 consecutive regions (a stride of 64 bytes) hit 8
// distinct 16-byte bank groups.  16 halo words after the row repeat its
// first 16 (windows that run past the row's end wrap there).
#pragma once

#include "ptx.h"

namespace arol {

constexpr int kRegionThreads = 128;

__device__ __forceinline__ int region_unit(int f) { return (f & ~3) | ((f & 3) ^ ((f >> 3) & 3)); }

// Stages the n words at xr (n a multiple of 16, xr 16-byte aligned) into xs
// swizzled, then the 16 halo words: 16-byte cp.async copies by the block's
// threads, completed by the caller's wait on its copy groups.
__device__ __forceinline__ void stage_region_row(float* xs, const float* xr, int n) {
    const int W4 = n >> 2;
    for (int f = threadIdx.x; f < W4 + 4; f += blockDim.x)
        ptx::cp_async16(xs + 4 * region_unit(f), xr + 4 * (f < W4 ? f : f - W4));
}

}  // namespace arol
