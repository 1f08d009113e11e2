// 2-D, FP64 kernels.
#define DGX_DIM 2
#define DGX_REAL double
#define DGX_SUFFIX 2d_f64
#define DGX_TILES(X) \
    X(0, 16, 8, 1, 16, 16, 1) X(1, 8, 8, 1, 16, 8, 1) X(2, 8, 4, 1, 16, 8, 1) \
    X(3, 4, 4, 1, 8, 8, 1) X(4, 4, 4, 1, 8, 4, 1) X(5, 4, 2, 1, 8, 4, 1)
#define DGX_STAGE_RUN run_stage2_any
#include "dgx_inst.cuh"
