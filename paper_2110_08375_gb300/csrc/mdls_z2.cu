// Instantiation of the complex md path for P = 2 limbs.
#include "zdriver.cuh"
MDLS_INSTANTIATE_Z(2)
