// plan.h -- choosing a kernel variant and tiling for one plot.
#pragma once

#include <cstdint>
#include <string>

#include "variants.h"

namespace ap {

struct Plan {
    const Variant *v = nullptr;
    int w = 0;            // window length (key window)
    int nu = 1, mu = 0;   // score blow-up {nu, mu, 0}; nu = 1 is LCS
    int64_t step = 1;     // vertical step: plot row r is the x-window at r * step
    int comb_rows = 0;    // physical comb height: nu * w
    int renorm = 0;       // steps between key renormalisations
    int ring = 0;         // exit-ring slots (power of two > w)
    int strips_per_warp = 0;
    int64_t rows = 0, cols = 0;
    int64_t chunk = 0, nchunks = 0, nsg = 0, ntiles = 0;
    size_t smem = 0;      // dynamic shared memory per block
    int warp_words = 0;   // shared-memory words per warp
    int max_value = 0;    // largest plot value: match * w = scale * nu * w
    int scale = 1;        // plot = scale x the combed (gcd-reduced) scheme's plot
};

// Picks the variant for window w and score blow-up {nu, mu, 0}.  `groups` > 0
// asks for that many threads per strip group (when a variant exists).
// Returns false (with a message) when no compiled variant covers the request.
// `lane_bits` > 0 asks for that lane format (8, 10 or 16 bits, LCS) where it
// covers the window.
bool choose_variant(int w, int nu, int mu, int groups, int64_t step, Plan *pl,
                    std::string *why, int lane_bits = 0);

// Tiles a rows x cols plot for the chosen variant.  `chunk_hint` > 0 forces
// the column chunk (rounded up to a multiple of 32).
void tile_plan(Plan *pl, int64_t rows, int64_t cols, int64_t chunk_hint, int device);

// Kernel parameters of one plot (shared by plain and batched launches).
void fill_params(const Plan &pl, const uint8_t *x, int64_t m, const uint8_t *y, int64_t n,
                 void *out, int out_bytes, int64_t ld, CombParams *p);

// Debug builds (AP_DEBUG_BOUNDS): the current device's word of bounds-check
// violation bits (allocated on first use); null in other builds.
uint32_t *debug_flags();

// Raises a kernel's dynamic shared-memory limit (once per kernel and device).
cudaError_t raise_smem_limit(const void *fn);

// Launch one comb over `pl` on `stream`.
cudaError_t launch_comb(const Plan &pl, const uint8_t *x, int64_t m, const uint8_t *y,
                        int64_t n, void *out, int out_bytes, int64_t ld, cudaStream_t stream);

// Physical comb cell updates for a plan (warm-up and padding included).
int64_t physical_cells(const Plan &pl);

// Match tables of a plan (used by warps whose x letters take at most four
// values): 0 none; 1 one thread per strip group; 2, 3 shared by G > 1
// threads, the row split rounded down (2) or up (3).
int plan_tables(const Plan &pl);

}  // namespace ap
