// Register plane kernels: the shapes of part 3 of PSATD_REG_SHAPES (reg_planes.cuh).
#define PSATD_PLANE_PART 3
#include "reg_planes.cuh"
