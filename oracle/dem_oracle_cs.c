/*
 * Complex-step build of the FP64 oracle's dynamics (test infrastructure only):
 * derivatives of rollouts with respect to E, e and mu, exact up to rounding,
 * used as the FP64 reference gradient.  See dem_oracle_dyn.h.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "dem_oracle_common.h"

#define OR_REAL 0
#include "dem_oracle_dyn.h"
