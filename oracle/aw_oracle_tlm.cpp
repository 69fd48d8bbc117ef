// Tangent-linear build of the oracle (TEST INFRASTRUCTURE): aw_oracle.c
// compiled with every double a dual number (oc_scalar.hpp).  Every entry point
// keeps its meaning; each floating-point argument or array element is a
// (value, tangent) pair, e.g. Q [n_tris][4][2].  Loading a state with seeded
// tangents and running sweeps gives the directional derivative of the sweep
// map along them; the values equal those of the plain build bit for bit.
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "oc_scalar.hpp"

#define double dual
#include "aw_oracle.c"
#undef double
