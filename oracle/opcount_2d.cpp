// ORACLE -- test and measurement infrastructure only: hwo_2d.c with the
// counting scalar of opcount.h (see opcount.cpp).
#include "opcount.h"

#define double hwo_real
#include "hweno_oracle.h"
#include "hwo_2d.c"
#undef double
