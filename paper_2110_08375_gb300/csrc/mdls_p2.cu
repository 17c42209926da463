// Instantiation of the plain md path for P = 2 limbs.
#include "driver.cuh"
MDLS_INSTANTIATE(2)
