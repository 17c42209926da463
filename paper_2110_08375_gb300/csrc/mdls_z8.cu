// Instantiation of the complex md path for P = 8 limbs.
#include "zdriver.cuh"
MDLS_INSTANTIATE_Z(8)
