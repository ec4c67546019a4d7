// ORACLE -- test and measurement infrastructure only (like the rest of this
// directory).
//
// Floating-point operation counts of the oracle's operator: the oracle's own C
// sources, unchanged, compiled as C++ with `double` replaced by a scalar that
// counts every addition, subtraction, multiplication, division and square
// root it performs (comparisons, fabs and copies are not counted).  A call of
// hwo1d_rhs / hwo2d_rhs on a grid of N cells with every cell smooth
// (HWO_TROUBLED_NONE) or every cell troubled (HWO_TROUBLED_ALL) gives the
// algorithmic flops of one cell-stage of Eq. (odeH) / Eq. (ode2) on each path
// (the Runge-Kutta combination of Eq. (RK) adds 2 flops per value per stage on
// top).  The arithmetic itself is the plain build's: each counted operation is
// one IEEE operation on doubles in the source's order, so the results are
// bitwise those of the plain (non-contracting) build.
#include "opcount.h"

unsigned long long hwo_ops[5];

#define double hwo_real
#include "hweno_oracle.h"  // before the source: its names keep their C linkage
#include "hwo_common.c"
#undef double

extern "C" {

// Operation counts [add/sub, mul, div, sqrt, pow] since the last reset.
void hwo_opcount_read(unsigned long long* out) {
  for (int k = 0; k < 5; ++k) out[k] = hwo_ops[k];
}
void hwo_opcount_reset(void) {
  for (int k = 0; k < 5; ++k) hwo_ops[k] = 0;
}

}  // extern "C"
