// Instantiation of the complex md path for P = 4 limbs.
#include "zdriver.cuh"
MDLS_INSTANTIATE_Z(4)
