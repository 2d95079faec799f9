// variants.h -- registry of compiled strip-comb kernel variants.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "comb.cuh"

namespace ap {

typedef void (*comb_fn_t)(CombParams);
typedef void (*batch_fn_t)(BatchParams);

struct Variant {
    int key_bits;    // 7 (8-bit lanes), 8 (8-bit lanes, full keys), 9 (10-bit lanes) or 15
    int lane_bits;   // 8, 10 or 16
    int rows;        // R: physical comb rows per thread
    int groups;      // G: threads per strip group
    int nu, mu;      // score blow-up {nu, mu, 0}; nu = 1 is LCS
    int xrows;       // 1: vertical-step layout (one x word per unit)
    int padu;        // trailing units of each thread that may be padding
    comb_fn_t fn;
    batch_fn_t batch_fn;
};

// Filled by the instantiation units (variants_*.cu).
const Variant *variant_table(int *count);

}  // namespace ap

// Instantiation helper: one template instance plus its registry entry.
#define AP_VARIANT(LANES, KEYBITS, BITS, R, G, NU, MU, PADU, XR)                    \
    { KEYBITS, BITS, R, G, NU, MU, XR, PADU, &ap::comb_kernel<ap::LANES, R, G, NU, MU, PADU, XR>, \
      &ap::comb_batch_kernel<ap::LANES, R, G, NU, MU, PADU, XR> }
