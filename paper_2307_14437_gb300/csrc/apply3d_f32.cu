// FP32 instantiation of the 3D product.
#define REAL float
#define AFD3D_FN afd_3d_f32
#define AFD3D_ATTR_FN afd_3d_attrs_f32
#include "apply3d_launch.cuh"
