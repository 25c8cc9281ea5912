// Register plane kernels: the shapes of part 1 of PSATD_REG_SHAPES (reg_planes.cuh).
#define PSATD_PLANE_PART 1
#include "reg_planes.cuh"
