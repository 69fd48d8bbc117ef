// Operation-counting build of the oracle (TEST INFRASTRUCTURE): aw_oracle.c
// compiled with every double an opcount (oc_scalar.hpp), which counts the
// floating-point operations of the oracle's own arithmetic, by phase of the
// sweep.  Floating-point arguments are plain doubles of the same layout.
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "oc_scalar.hpp"

int64_t oc_flops[OC_PH_N];
int oc_phase = OC_PH_OTHER;

#define OC_PHASE(p) (oc_phase = (p))
#define double opcount
#include "aw_oracle.c"
#undef double

// operations counted so far by phase (other, node solver, fluxes, FV update,
// reconstruction, local step, predictor); reset sets them to zero
extern "C" void oc_count_read(int64_t* out) {
  for (int k = 0; k < OC_PH_N; ++k) out[k] = oc_flops[k];
}
extern "C" void oc_count_reset(void) {
  for (int k = 0; k < OC_PH_N; ++k) oc_flops[k] = 0;
}
