// FP64 instantiation of the 3D product.
#define REAL double
#define AFD3D_FN afd_3d_f64
#define AFD3D_ATTR_FN afd_3d_attrs_f64
#include "apply3d_launch.cuh"
