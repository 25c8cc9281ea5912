// Register plane kernels: the shapes of part 0 of PSATD_REG_SHAPES (reg_planes.cuh).
#define PSATD_PLANE_PART 0
#include "reg_planes.cuh"
