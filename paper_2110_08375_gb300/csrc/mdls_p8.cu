// Instantiation of the plain md path for P = 8 limbs.
#include "driver.cuh"
MDLS_INSTANTIATE(8)
