// Double-float instantiation of the 3D product: FP64 inputs, weights, symbol
// and outputs, the FFTs and the symbol product in double-float arithmetic
// (about 48 bits), for the FP64 residual of the mixed solver at FP32 rates.
#define REAL dfl
#define AFD3D_FN afd_3d_df
#define AFD3D_ATTR_FN afd_3d_attrs_df
#include "apply3d_launch.cuh"
