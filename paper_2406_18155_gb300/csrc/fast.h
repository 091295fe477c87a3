// Fast evolution paths (on-chip per-column kernels and the tiled slab kernels).
#pragma once
#include "kplan.h"

// True when the on-chip kernel can evolve this plan (every column block fits in
// shared memory).
bool fast_onchip_available(const KPlan& p, bool mixed);
// Evolves psi (D x S complex128, column innermost) through N RK4 steps in place,
// stage tables `tab` (complex64 rows when mixed, complex128 otherwise).
sg_status fast_onchip_forward(sg_system* sys, const KPlan& p, bool mixed, const void* tab,
                              double2* psi, int N, double dt, cudaStream_t st, int* launches);
