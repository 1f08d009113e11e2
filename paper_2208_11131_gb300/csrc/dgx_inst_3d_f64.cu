// 3-D, FP64 kernels.
#define DGX_DIM 3
#define DGX_REAL double
#define DGX_SUFFIX 3d_f64
#define DGX_TILES(X) \
    X(0, 4, 4, 4, 8, 4, 4) X(1, 4, 2, 2, 4, 4, 4) X(2, 2, 2, 2, 4, 4, 2) \
    X(3, 2, 2, 1, 4, 2, 2) X(4, 2, 1, 1, 2, 2, 2) X(5, 1, 1, 1, 2, 2, 1)
#define DGX_STAGE_RUN run_stage2_any
#include "dgx_inst.cuh"
