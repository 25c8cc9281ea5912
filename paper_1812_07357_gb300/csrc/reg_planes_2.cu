// Register plane kernels: the shapes of part 2 of PSATD_REG_SHAPES (reg_planes.cuh).
#define PSATD_PLANE_PART 2
#include "reg_planes.cuh"
