// FP32 instantiation of the transposed-spectrum 2D product.
#define REAL float
#define AFD2D_FN afd_2d_f32
#define AFD2D_ATTR_FN afd_2d_attrs_f32
#include "apply2d_launch.cuh"
