// FP64 instantiation of the transposed-spectrum 2D product.
#define REAL double
#define AFD2D_FN afd_2d_f64
#define AFD2D_ATTR_FN afd_2d_attrs_f64
#include "apply2d_launch.cuh"
