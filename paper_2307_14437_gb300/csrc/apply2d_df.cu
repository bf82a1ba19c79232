// Double-float instantiation of the transposed-spectrum 2D product: FP64
// inputs, weights, symbol and outputs, the FFTs and the symbol product in
// double-float arithmetic (about 48 bits), for the FP64 residual of the mixed
// solver at FP32 arithmetic rates.
#define REAL dfl
#define AFD2D_FN afd_2d_df
#define AFD2D_ATTR_FN afd_2d_attrs_df
#include "apply2d_launch.cuh"
