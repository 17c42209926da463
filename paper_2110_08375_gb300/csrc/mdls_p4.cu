// Instantiation of the plain md path for P = 4 limbs.
#include "driver.cuh"
MDLS_INSTANTIATE(4)
